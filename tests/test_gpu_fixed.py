"""GPU tests of the exact fixed-point path (AMR_PREC_FIXED) and of the
full-size configurations, through the C ABI, against the FP64 oracle.

The fixed-point path rounds each staged coarse value once onto a grid of
2^-47 of the region's largest magnitude per unknown and is exact integer
arithmetic afterwards, so it is held to the float64 tolerance (1e-12
normwise per item and unknown).  The full-size tests sample outputs of the
20,000-item uneven batch (autotuned, graph captured) and of the 8,192-face
puncture batch and compare them one by one with the oracle's single-output
evaluators.
"""
import numpy as np
import pytest
import torch

from oracle import transfer as tr
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import gpu_interpolate, gpu_restrict, normwise_errors, record, written_masks

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SPLIT_BOUND = 2e-6


def _faces(U, order, seed, p=6, k=3):
    n = 6
    items, cl, fl = wl.make_items(list(range(6)), [-1] * n, [p] * n, [k] * n, [order] * n, U)
    rng = np.random.Generator(np.random.PCG64(wl.SEED_BASE + 500 + seed))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(n, rng))
    return items, coarse.numpy(), fine.numpy()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_fixed_magnitudes_per_unknown(order):
    """Unknowns spanning 1e-280 .. 1e300, zeros, a constant power of two and
    a large constant with a 1e-12 variation: each unknown has its own grid,
    so every one stays within the float64 tolerance."""
    U = 8
    items, c, f = _faces(U, order, order)
    scales = np.array([1.0, 1e300, 1e-280, 0.0, 0.0, 1e-8, 1.0, 3.5e5])
    c = (c.reshape(-1, U) * scales).copy()
    f = (f.reshape(-1, U) * scales).copy()
    c[:, 4] = f[:, 4] = 2.0 ** 10
    c[:, 6] = 1.0 + 1e-12 * c[:, 6]
    f[:, 6] = 1.0 + 1e-12 * f[:, 6]
    c, f = c.reshape(-1), f.reshape(-1)
    plan = B.Plan(items, U, len(c), len(f), B.PREC_FIXED)
    fm, cm = written_masks(items, U, len(c), len(f))
    f_ref, c_ref = tr.interpolate(items, U, c, f), tr.restrict(items, U, f, c)
    f_gpu, c_gpu = gpu_interpolate(plan, c, f), gpu_restrict(plan, f, c)
    e_i, _ = normwise_errors(items, U, f_gpu, f_ref, fm, "fine")
    e_r, _ = normwise_errors(items, U, c_gpu, c_ref, cm, "coarse")
    record(test="fixed_magnitudes", order=order, interp=e_i, restrict=e_r)
    assert e_i <= FP64_TOL and e_r <= FP64_TOL, (e_i, e_r)
    # zeros stay exact zeros; a constant is exact up to the rounding of the
    # centre value onto the grid (2^-48 of it)
    g = f_gpu.reshape(-1, U)[fm.reshape(-1, U)[:, 3], 3]
    assert np.all(g == 0.0)
    g = f_gpu.reshape(-1, U)[fm.reshape(-1, U)[:, 4], 4]
    assert np.abs(g - 2.0 ** 10).max() <= 1e-14 * 2.0 ** 10
    plan.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_fixed_non_finite_inputs(order):
    """A NaN or an infinity in one unknown's stencil region of one face makes
    every non-injected child of that unknown on that face NaN (a superset of
    the outputs the oracle makes non-finite); injected children are copies;
    other unknowns and faces are unaffected."""
    U = 4
    items, c, f = _faces(U, order, 10 + order)
    arr = 2 * 3 * 36 * U
    c = c.copy()
    # face 2, unknown 1: a NaN in the coarse layer next to the interface;
    # face 4, unknown 2: +inf there
    for item, u, val in ((2, 1, np.nan), (4, 2, np.inf)):
        co = int(items[item]["coarse_offset"])
        c[co + (3 * 36 + 2 * 6 + 2) * U + u] = val  # some volume of the face array
    plan = B.Plan(items, U, len(c), len(f), B.PREC_FIXED)
    fm, _ = written_masks(items, U, len(c), len(f))
    f_ref = tr.interpolate(items, U, c, f)
    f_gpu = gpu_interpolate(plan, c, f)
    for i, it in enumerate(items):
        fo = int(it["fine_offset"])
        g = f_gpu[fo:fo + 9 * arr].reshape(-1, U)
        r = f_ref[fo:fo + 9 * arr].reshape(-1, U)
        m = fm[fo:fo + 9 * arr].reshape(-1, U)
        for u in range(U):
            sel = m[:, u]
            bad = (i, u) in ((2, 1), (4, 2))
            if not bad:
                scale = np.abs(r[sel, u]).max()
                assert np.abs(g[sel, u] - r[sel, u]).max() <= FP64_TOL * scale
                continue
            # the children left finite are the injected ones, one per coarse
            # centre (36 on a p = 6 face), copies of the centre values
            gs, rs = g[sel, u], r[sel, u]
            fin = ~np.isnan(gs)
            assert np.count_nonzero(fin) == 36
            assert np.all((gs[fin] == rs[fin]) | ~np.isfinite(rs[fin]))
    plan.close()


@pytest.mark.parametrize("order", [2, 3])
def test_fixed_reproduces_polynomials(order):
    """Taylor-m reproduces polynomials of degree m exactly (Sec. 3); the
    fixed-point path does so up to the quantization, 1e-13 of the field."""
    U = 1
    items, cl, fl = wl.make_items(list(range(6)), [-1] * 6, [9] * 6, [3] * 6, [order] * 6, U)
    rng = np.random.default_rng(40 + order)
    coef = rng.uniform(-1, 1, (4, 4, 4))
    H = 1.0 / 9

    def poly(x):
        x = x * H
        out = torch.zeros_like(x[:, 0])
        for a in range(order + 1):
            for b in range(order + 1 - a):
                for d in range(order + 1 - a - b):
                    out = out + float(coef[a, b, d]) * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** d
        return out[:, None]

    coarse, fine = wl.polynomial_buffers(items, U, cl, fl, poly, origins=rng.uniform(-20, 20, (6, 3)))
    c, f = coarse.numpy(), fine.numpy()
    plan = B.Plan(items, U, cl, fl, B.PREC_FIXED)
    fm, _ = written_masks(items, U, cl, fl)
    f_gpu = gpu_interpolate(plan, c, f)
    assert np.abs(f_gpu[fm] - f[fm]).max() <= 1e-13 * np.abs(c).max()
    plan.close()


def test_split_non_finite_and_out_of_range():
    """Split precision: a NaN input propagates as NaN (not as an infinity),
    and values of 2^128 or more give non-finite results, as documented."""
    U = 2
    items, c, f = _faces(U, 3, 20)
    c = c.copy()
    co = int(items[0]["coarse_offset"])
    c[co + (2 * 36 + 2 * 6 + 2) * U + 0] = np.nan
    c.reshape(-1, U)[int(items[1]["coarse_offset"]) // U:(int(items[1]["coarse_offset"]) + 216 * U) // U, 1] = 1e300
    plan = B.Plan(items, U, len(c), len(f), B.PREC_SPLIT)
    fm, _ = written_masks(items, U, len(c), len(f))
    f_ref = tr.interpolate(items, U, c, f)
    f_gpu = gpu_interpolate(plan, c, f)
    arr = 2 * 3 * 36 * U
    fo = int(items[0]["fine_offset"])
    g, r = f_gpu[fo:fo + 9 * arr].reshape(-1, U), f_ref[fo:fo + 9 * arr].reshape(-1, U)
    m = fm[fo:fo + 9 * arr].reshape(-1, U)[:, 0]
    gs = g[m, 0]
    # the NaN reaches outputs as NaN, never as an infinity
    assert np.isnan(gs).any() and not np.isinf(gs).any()
    assert np.isnan(r[m, 0]).any()
    fo = int(items[1]["fine_offset"])
    g = f_gpu[fo:fo + 9 * arr].reshape(-1, U)
    m = fm[fo:fo + 9 * arr].reshape(-1, U)[:, 1]
    gs = g[m, 1]
    # every child but the injected copies (one per centre) is non-finite
    assert np.count_nonzero(np.isfinite(gs)) == 36 and np.all(gs[np.isfinite(gs)] == 1e300)
    plan.close()


def _owned(s, p):
    return (s * p + 1) // 3, (s * p + p + 1) // 3


def _sample_check(items, U, coarse, fine, f_out, c_out, n_items, per_item, seed):
    """Worst normwise error of sampled ghost and halo outputs against the
    oracle's single-output evaluators; scale = the larger of max|coarse| and
    max|fine| of that item and unknown."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for i in rng.choice(len(items), n_items, replace=False):
        it = items[int(i)]
        face, sub = int(it["face"]), int(it["subface"])
        p, k = int(it["patch_size"]), int(it["overlap"])
        n_ax = face % 3
        arr = 2 * k * p * p * U
        nsub = 9 if sub < 0 else 1
        co, fo = int(it["coarse_offset"]), int(it["fine_offset"])
        c_it = coarse[co:co + arr].cpu().numpy()
        f_it = fine[fo:fo + nsub * arr].cpu().numpy()
        loc = it.copy()
        loc["coarse_offset"], loc["fine_offset"] = 0, 0
        scale = np.maximum(np.abs(c_it.reshape(-1, U)).max(0), np.abs(f_it.reshape(-1, U)).max(0))
        ext = [p, p, p]
        ext[n_ax] = 2 * k
        _, t0, t1 = [n_ax] + [d for d in range(3) if d != n_ax]
        idx_g, idx_h = [], []
        for _ in range(per_item):
            u = int(rng.integers(U))
            slot = int(rng.integers(nsub))
            j = int(rng.integers(1, k + 1))
            idx = [int(rng.integers(p)) for _ in range(3)]
            idx[n_ax] = k - j if face < 3 else k - 1 + j
            vol = (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]
            idx_g.append((slot * arr + vol * U + u, u))
            # a coarse halo volume this item restricts
            s = int(rng.integers(9)) if sub < 0 else sub
            idx = [0, 0, 0]
            for ax, st in ((t0, s % 3), (t1, s // 3)):
                lo, hi = _owned(st, p)
                idx[ax] = int(rng.integers(lo, hi))
            jj = int(rng.integers(k))
            idx[n_ax] = k + jj if face < 3 else k - 1 - jj
            vol = (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]
            idx_h.append((vol * U + u, u))
        got_g = f_out[torch.tensor([fo + e for e, _ in idx_g], device=f_out.device)].cpu().numpy()
        got_h = c_out[torch.tensor([co + e for e, _ in idx_h], device=c_out.device)].cpu().numpy()
        for (e, u), g in zip(idx_g, got_g):
            worst = max(worst, abs(g - tr.interpolate_one(loc, U, c_it, e)) / max(scale[u], 1e-300))
        for (e, u), g in zip(idx_h, got_h):
            worst = max(worst, abs(g - tr.restrict_one(loc, U, f_it, e)) / max(scale[u], 1e-300))
    return worst


@pytest.mark.parametrize("precision,tol", [(B.PREC_FIXED, FP64_TOL), (B.PREC_FP64, FP64_TOL)])
def test_full_size_uneven_batch_autotuned_graph(precision, tol):
    """20,000 subface items, p 6/9/12, k 2/3, orders 1/2/3, U = 59: the
    autotuned, graph-captured step against the oracle on sampled outputs."""
    items, coarse, fine = wl.uneven_batch(device="cuda")
    U = 59
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), precision)
    plan.autotune(coarse, fine.clone(), coarse.clone())
    f_out, c_out = fine.clone(), coarse.clone()
    plan.capture_step(coarse, f_out, c_out)
    plan.launch_step()
    torch.cuda.synchronize()
    # restriction read the interpolated ghosts: compare it against the oracle
    # on the same (interpolated) fine data
    worst = _sample_check(items, U, coarse, f_out, f_out, c_out, 150, 10, seed=3)
    record(test="full_size_uneven", precision=precision, worst=worst)
    assert worst <= tol, worst
    plan.close()


@pytest.mark.parametrize("precision,tol", [(B.PREC_FIXED, FP64_TOL), (B.PREC_FP64, FP64_TOL),
                                           (B.PREC_SPLIT, SPLIT_BOUND)])
def test_full_size_puncture_batch(precision, tol):
    """8,192 hanging faces, p = 9, k = 3, U = 59, Taylor-3, puncture-like
    fields (psi = 1 + M / 2r clipped at r = H/2, lapse- and shift-like
    fields): sampled outputs against the oracle."""
    items, coarse, fine = wl.puncture_batch(device="cuda")
    U = 59
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), precision)
    plan.autotune(coarse, fine.clone(), coarse.clone())
    f_out, c_out = fine.clone(), coarse.clone()
    plan.interpolate(coarse, f_out)
    plan.restrict(fine, c_out)
    torch.cuda.synchronize()
    worst = _sample_check(items, U, coarse, fine, f_out, c_out, 120, 12, seed=4)
    record(test="full_size_puncture", precision=precision, worst=worst)
    assert worst <= tol, worst
    plan.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_fixed_restriction_windows(order):
    """Restriction of fixed-point plans (float64 columns and exact integer
    columns side by side) on adversarial windows: unknowns scaled to both
    sides of both ends of the integer path's range (2^-923 .. 2^977), values
    spread over twenty decades inside one window, a NaN in one fine face
    array; every unknown matches the oracle at the float64 tolerance (NaN
    where the oracle gives NaN)."""
    U = 8
    items, c, f = _faces(U, order, 30 + order, p=9)
    rng = np.random.default_rng(77 + order)
    scales = np.array([1.0, 2.0 ** -922, 2.0 ** -925, 2.0 ** 975, 2.0 ** 978, 1.0, 3.5e5, 1.0])
    f = (f.reshape(-1, U) * scales).copy()
    f[:, 5] *= 10.0 ** rng.uniform(-20.0, 0.0, len(f))
    fo = int(items[3]["fine_offset"])
    f[fo // U:fo // U + 2 * 3 * 81, 7] = np.nan  # face 3, unknown 7: the first fine face array
    f = f.reshape(-1)
    plan = B.Plan(items, U, len(c), len(f), B.PREC_FIXED)
    _, cm = written_masks(items, U, len(c), len(f))
    c_ref = tr.restrict(items, U, f, c)
    c_gpu = gpu_restrict(plan, f, c)
    plan.close()
    assert np.array_equal(np.isnan(c_gpu[cm]), np.isnan(c_ref[cm]))
    assert np.isnan(c_ref[cm]).any()
    ok = cm & ~np.isnan(c_ref)
    e_r, rms = normwise_errors(items, U, c_gpu, c_ref, ok, "coarse")
    record(test="fixed_restriction_windows", order=order, restrict=e_r, rms=rms)
    assert e_r <= FP64_TOL, e_r
