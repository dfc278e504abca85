"""Adjoint parity on the GPU: P^T and R^T (through the C ABI) against the
oracle's explicit transposes, the dot-product identity with the GPU forward
operators, and the autograd Functions against central finite differences."""
import numpy as np
import pytest
import torch

from oracle import transfer as tr
from paper_2504_15814_gb300 import autograd as AG
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import record

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _shared_batch(order, p, k, U):
    """Nine subface items sharing one coarse face array, plus whole faces of
    every orientation with private arrays."""
    arr = 2 * k * p * p * U
    items = np.zeros(9 + 6, dtype=wl.ITEM_DTYPE)
    for s in range(9):
        items[s] = (2, s, p, k, order, 0, 0, s * arr)
    for f in range(6):
        items[9 + f] = (f, -1, p, k, order, 0, (1 + f) * arr, 9 * arr + f * 9 * arr)
    return items, 7 * arr, 9 * arr + 6 * 9 * arr


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("order,k", [(1, 1), (1, 3), (2, 2), (2, 3), (3, 2), (3, 3)])
@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_SPLIT, B.PREC_FIXED])
def test_adjoints_match_oracle_transposes(order, k, precision):
    p, U = 6, 5
    items, cl, fl = _shared_batch(order, p, k, U)
    rng = np.random.default_rng(order * 10 + k)
    g_f, g_c = rng.standard_normal(fl), rng.standard_normal(cl)
    plan = B.Plan(items, U, cl, fl, precision)
    out_c = torch.full((cl,), np.nan, dtype=torch.float64, device="cuda")
    plan.interpolate_adjoint(torch.as_tensor(g_f).cuda(), out_c)
    out_f = torch.full((fl,), np.nan, dtype=torch.float64, device="cuda")
    plan.restrict_adjoint(torch.as_tensor(g_c).cuda(), out_f)
    torch.cuda.synchronize()
    ref_c = tr.interpolate_adjoint(items, U, g_f, cl)
    ref_f = tr.restrict_adjoint(items, U, g_c, fl)
    e1, e2 = _rel(out_c.cpu().numpy(), ref_c), _rel(out_f.cpu().numpy(), ref_f)
    record(test="adjoint_vs_oracle", order=order, k=k, precision=precision, pt=e1, rt=e2)
    assert e1 <= TOL and e2 <= TOL, (e1, e2)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_dot_product_identity(order):
    U = 7
    n = 12
    items, cl, fl = wl.make_items([i % 6 for i in range(n)], [-1] * n, [9] * n, [3] * n, [order] * n, U)
    plan = B.Plan(items, U, cl, fl, B.PREC_FP64)
    g = torch.Generator(device="cuda").manual_seed(order)
    v_c = torch.randn(cl, dtype=torch.float64, device="cuda", generator=g)
    v_f = torch.randn(fl, dtype=torch.float64, device="cuda", generator=g)
    g_f = torch.randn(fl, dtype=torch.float64, device="cuda", generator=g)
    g_c = torch.randn(cl, dtype=torch.float64, device="cuda", generator=g)
    Pv = torch.zeros(fl, dtype=torch.float64, device="cuda")
    plan.interpolate(v_c, Pv)
    PTg = torch.empty(cl, dtype=torch.float64, device="cuda")
    plan.interpolate_adjoint(g_f, PTg)
    Rv = torch.zeros(cl, dtype=torch.float64, device="cuda")
    plan.restrict(v_f, Rv)
    RTg = torch.empty(fl, dtype=torch.float64, device="cuda")
    plan.restrict_adjoint(g_c, RTg)
    a, b = float(torch.dot(g_f, Pv)), float(torch.dot(PTg, v_c))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b) + 1e-300) * 10
    a, b = float(torch.dot(g_c, Rv)), float(torch.dot(RTg, v_f))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b) + 1e-300) * 10


def _fd_check(items, coarse, fine, U, n_dirs, h=1e-6, seed=0):
    """Gradient of L = <G1, Interpolate(c, f)> + <G2, Restrict(f, c)> through
    autograd against central differences along random unit directions.

    L is linear, so the central difference is exact up to the float64 rounding
    of L itself, at most ~eps * S with S = sum |G1||Interpolate| + sum
    |G2||Restrict|; the check allows 64 eps S / (2h) and returns the largest
    |fd - analytic| as a fraction of that bound."""
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), B.PREC_FP64)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    G1 = torch.randn(fine.numel(), dtype=torch.float64, device="cuda", generator=gen)
    G2 = torch.randn(coarse.numel(), dtype=torch.float64, device="cuda", generator=gen)

    def loss(c, f):
        return torch.dot(G1, AG.interpolate(c, f, plan)) + torch.dot(G2, AG.restrict(f, c, plan))

    c = coarse.clone().requires_grad_(True)
    f = fine.clone().requires_grad_(True)
    loss(c, f).backward()
    with torch.no_grad():
        S = float(torch.dot(G1.abs(), AG.interpolate(coarse, fine, plan).abs())
                  + torch.dot(G2.abs(), AG.restrict(fine, coarse, plan).abs()))
    bound = 64 * 2.220446049250313e-16 * S / (2 * h)
    worst = 0.0
    for _ in range(n_dirs):
        dc = torch.randn(coarse.numel(), dtype=torch.float64, device="cuda", generator=gen)
        df = torch.randn(fine.numel(), dtype=torch.float64, device="cuda", generator=gen)
        nrm = torch.sqrt(torch.dot(dc, dc) + torch.dot(df, df))
        dc, df = dc / nrm, df / nrm
        with torch.no_grad():
            fd = (loss(coarse + h * dc, fine + h * df) - loss(coarse - h * dc, fine - h * df)) / (2 * h)
        an = torch.dot(c.grad, dc) + torch.dot(f.grad, df)
        worst = max(worst, float(abs(fd - an)) / bound)
    plan.close()
    return worst


def test_autograd_finite_differences_small():
    items, coarse, fine = wl.uniform_batch(n_faces=24, U=59, order=3, config_index=4, device="cuda")
    worst = _fd_check(items, coarse, fine, 59, 16)
    record(test="autograd_fd_small", fraction_of_rounding_bound=worst)
    assert worst <= 1.0, worst


def test_adjoint_full_size_sampled():
    """4,096 hanging faces, p = 9, k = 3, U = 59, Taylor-3: autograd gradient
    against central differences (h = 1e-6) on 64 random directions, and P^T /
    R^T of 32 sampled faces against the oracle's explicit transposes."""
    U = 59
    items, coarse, fine = wl.uniform_batch(n_faces=4096, U=U, order=3, config_index=4, device="cuda")
    worst = _fd_check(items, coarse, fine, U, 64)
    record(test="autograd_fd_full", fraction_of_rounding_bound=worst)
    assert worst <= 1.0, worst
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), B.PREC_FP64)
    gen = torch.Generator(device="cuda").manual_seed(9)
    gf = torch.randn(fine.numel(), dtype=torch.float64, device="cuda", generator=gen)
    gc = torch.randn(coarse.numel(), dtype=torch.float64, device="cuda", generator=gen)
    oc = torch.empty_like(gc)
    of = torch.empty_like(gf)
    plan.interpolate_adjoint(gf, oc)
    plan.restrict_adjoint(gc, of)
    torch.cuda.synchronize()
    arr = 2 * 3 * 81 * U
    rng = np.random.default_rng(3)
    worst = 0.0
    for i in rng.choice(len(items), 32, replace=False):
        it = items[int(i)].copy()
        co, fo = int(it["coarse_offset"]), int(it["fine_offset"])
        one = np.array([it])
        one["coarse_offset"], one["fine_offset"] = 0, 0
        ref_c = tr.interpolate_adjoint(one, U, gf[fo:fo + 9 * arr].cpu().numpy(), arr)
        ref_f = tr.restrict_adjoint(one, U, gc[co:co + arr].cpu().numpy(), 9 * arr)
        worst = max(worst, _rel(oc[co:co + arr].cpu().numpy(), ref_c), _rel(of[fo:fo + 9 * arr].cpu().numpy(), ref_f))
    record(test="adjoint_full_sampled", worst=worst)
    assert worst <= TOL, worst
    plan.close()
