"""Batching machinery on the GPU: launch-shape tuning, the autotuner and the
captured step graph keep oracle parity (through the C ABI)."""
import numpy as np
import pytest
import torch

from oracle import transfer as tr
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import normwise_errors, written_masks

pytestmark = pytest.mark.gpu


def _batch(n=9, U=13, seed=1):
    rng = np.random.default_rng(seed)
    ps = rng.choice([6, 9, 12], n)
    ks = rng.choice([2, 3], n)
    orders = rng.choice([1, 2, 3], n)
    subs = rng.integers(-1, 9, n)
    items, cl, fl = wl.make_items(rng.integers(0, 6, n), subs, ps, ks, orders, U)
    g = np.random.Generator(np.random.PCG64(seed))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, g), wl.origins_in_box(n, g))
    return items, coarse.numpy(), fine.numpy()


def _check(items, U, c, f, f_gpu, c_gpu, tol):
    """Each operator against the oracle on the same original inputs:
    f_gpu = P applied to (c, f), c_gpu = R applied to (f, c)."""
    f_ref = tr.interpolate(items, U, c, f)
    c_ref = tr.restrict(items, U, f, c)
    fm, cm = written_masks(items, U, len(c), len(f))
    assert normwise_errors(items, U, f_gpu, f_ref, fm, "fine")[0] <= tol
    assert normwise_errors(items, U, c_gpu, c_ref, cm, "coarse")[0] <= tol


def _operators(plan, c, f):
    """Interpolation of (c, f) and restriction of the original (f, c) on the GPU."""
    cd, fd = torch.as_tensor(c).cuda(), torch.as_tensor(f).cuda()
    co = cd.clone()
    plan.interpolate(cd, fd)
    plan.restrict(torch.as_tensor(f).cuda(), co)
    torch.cuda.synchronize()
    return fd.cpu().numpy(), co.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(B.PREC_FP64, 1e-12), (B.PREC_SPLIT, 2e-6), (B.PREC_FIXED, 1e-12)])
@pytest.mark.parametrize("shape", [(128, 8192, 128, 0, 0), (256, 24 * 1024, 64, 1, 0), (64, 100 * 1024, 256, 3, 0),
                                   (256, 64 * 1024, 256, 2, 0), (256, 112 * 1024, 128, 2, 32),
                                   (64, 16 * 1024, 256, 1, 32), (384, 64 * 1024, 256, 3, 32)])
def test_set_tuning_keeps_parity(shape, precision, tol):
    U = 13
    items, c, f = _batch(U=U)
    plan = B.Plan(items, U, len(c), len(f), precision)
    if precision != B.PREC_SPLIT and shape[0] > 256:  # float64 and fixed-point CTAs hold at most 256 threads
        with pytest.raises(B.AmrError):
            plan.set_tuning(*shape)
        return
    plan.set_tuning(*shape)
    assert plan.tuning == dict(interp_threads=shape[0], interp_smem_budget=shape[1], restrict_threads=shape[2],
                               interp_addback=shape[3], interp_lanes=shape[4])
    _check(items, U, c, f, *_operators(plan, c, f), tol)


def test_invalid_tuning_rejected():
    items, c, f = _batch(n=2)
    plan = B.Plan(items, 13, len(c), len(f))  # float64: 384 threads is beyond its CTA limit
    for bad in [(16, 32768, 128), (256, 1024, 128), (256, 32768, 300), (512, 32768, 128), (256, 32768, 128, 4),
                (256, 32768, 128, 2, 16), (384, 32768, 128, 2, 32)]:
        with pytest.raises(B.AmrError):
            plan.set_tuning(*bad)


@pytest.mark.parametrize("precision,tol", [(B.PREC_FP64, 1e-12), (B.PREC_SPLIT, 2e-6), (B.PREC_FIXED, 1e-12)])
def test_autotune_and_step_graph(precision, tol):
    U = 13
    items, c, f = _batch(n=12, U=U, seed=4)
    plan = B.Plan(items, U, len(c), len(f), precision)
    cd = torch.as_tensor(c).cuda()
    fd = torch.as_tensor(f).cuda()
    co = cd.clone()
    chosen = plan.autotune(cd, fd, co)
    assert chosen == plan.tuning
    # the chosen shape keeps parity with the oracle
    _check(items, U, c, f, *_operators(plan, c, f), tol)
    # the step graph replays interpolate + restrict on the captured buffers:
    # the same results, bit for bit, as the two calls made directly
    fd.copy_(torch.as_tensor(f))
    co.copy_(cd)
    plan.capture_step(cd, fd, co)
    for _ in range(2):
        plan.launch_step()
    f2, c2 = torch.as_tensor(f).cuda(), cd.clone()
    for _ in range(2):
        plan.interpolate(cd, f2)
        plan.restrict(f2, c2)
    torch.cuda.synchronize()
    assert torch.equal(fd, f2) and torch.equal(co, c2)


def test_launch_without_capture_rejected():
    items, c, f = _batch(n=2)
    plan = B.Plan(items, 13, len(c), len(f))
    with pytest.raises(B.AmrError):
        plan.launch_step()


@pytest.mark.parametrize("precision", [B.PREC_SPLIT, B.PREC_FP64])
def test_warp_per_centre_mapping_is_bitwise_identical(precision):
    """interp_lanes = 32 (one warp per coarse centre, tiles of at most 32
    unknowns) changes only which thread computes a (centre, unknown) task,
    so with U = 59 (chunks of 30 and 29) and patch sizes that are and are not
    multiples of 3 its ghosts equal the dense mapping's bit for bit, and
    match the oracle."""
    U = 59
    rng = np.random.default_rng(23)
    n = 10
    ps = [9, 8, 6, 10, 12, 7, 9, 5, 24, 4]
    items, cl, fl = wl.make_items(rng.integers(0, 6, n), rng.integers(-1, 9, n), ps, rng.choice([2, 3], n),
                                  rng.choice([1, 2, 3], n), U)
    g = np.random.Generator(np.random.PCG64(29))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, g), wl.origins_in_box(n, g))
    cd = coarse.cuda()
    outs = []
    threads = 384 if precision == B.PREC_SPLIT else 256
    for shape in ((256, 64 * 1024, 256, 2, 0), (threads, 112 * 1024, 256, 2, 32), (256, 24 * 1024, 128, 2, 32)):
        plan = B.Plan(items, U, cl, fl, precision)
        plan.set_tuning(*shape)
        fd = fine.cuda().clone()
        plan.interpolate(cd, fd)
        torch.cuda.synchronize()
        outs.append(fd.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    c, f = coarse.numpy(), fine.numpy()
    fm, _ = written_masks(items, U, cl, fl)
    tol = 1e-12 if precision == B.PREC_FP64 else 2e-6
    assert normwise_errors(items, U, outs[1], tr.interpolate(items, U, c, f), fm, "fine")[0] <= tol


def test_pinned_host_buffers_match_device_buffers():
    """The kernels accept buffers in pinned host memory (read and written in
    place over the host link): same results, bit for bit, as on device
    buffers, for interpolate, restrict and a split-precision mixed batch."""
    U = 13
    items, c, f = _batch(n=9, U=U, seed=6)
    plan = B.Plan(items, U, len(c), len(f), B.PREC_SPLIT)
    cd, fd = torch.as_tensor(c).cuda(), torch.as_tensor(f).cuda()
    cod = cd.clone()
    plan.interpolate(cd, fd)
    plan.restrict(fd, cod)
    ch, fh = torch.as_tensor(c).pin_memory(), torch.as_tensor(f).pin_memory()
    coh = ch.clone().pin_memory()
    plan.interpolate(ch, fh)
    plan.restrict(fh, coh)
    torch.cuda.synchronize()
    assert torch.equal(fd.cpu(), fh) and torch.equal(cod.cpu(), coh)
    with pytest.raises(TypeError):
        plan.interpolate(torch.as_tensor(c), fh)  # pageable host memory is refused by the binding
