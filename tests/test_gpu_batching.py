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
    """Each operator against the oracle on the same inputs: interpolation on
    the original data, restriction on the fine buffer the GPU step produced
    (restriction reads the interpolated ghost layers, and Taylor
    extrapolation would amplify their split-precision error)."""
    f_ref = tr.interpolate(items, U, c, f)
    c_ref = tr.restrict(items, U, f_gpu, c)
    fm, cm = written_masks(items, U, len(c), len(f))
    assert normwise_errors(items, U, f_gpu, f_ref, fm, "fine")[0] <= tol
    assert normwise_errors(items, U, c_gpu, c_ref, cm, "coarse")[0] <= tol


@pytest.mark.parametrize("precision,tol", [(B.PREC_FP64, 1e-12), (B.PREC_SPLIT, 2e-6)])
@pytest.mark.parametrize("shape", [(128, 8192, 128, 0), (256, 24 * 1024, 64, 1), (64, 100 * 1024, 256, 3),
                                   (256, 64 * 1024, 256, 2)])
def test_set_tuning_keeps_parity(shape, precision, tol):
    U = 13
    items, c, f = _batch(U=U)
    plan = B.Plan(items, U, len(c), len(f), precision)
    plan.set_tuning(*shape)
    assert plan.tuning == dict(interp_threads=shape[0], interp_smem_budget=shape[1], restrict_threads=shape[2],
                               interp_addback=shape[3])
    cd, fd = torch.as_tensor(c).cuda(), torch.as_tensor(f).cuda()
    co = cd.clone()
    plan.interpolate(cd, fd)
    plan.restrict(fd, co)
    torch.cuda.synchronize()
    _check(items, U, c, f, fd.cpu().numpy(), co.cpu().numpy(), tol)


def test_invalid_tuning_rejected():
    items, c, f = _batch(n=2)
    plan = B.Plan(items, 13, len(c), len(f))
    for bad in [(16, 32768, 128), (256, 1024, 128), (256, 32768, 300), (512, 32768, 128), (256, 32768, 128, 4)]:
        with pytest.raises(B.AmrError):
            plan.set_tuning(*bad)


@pytest.mark.parametrize("precision,tol", [(B.PREC_FP64, 1e-12), (B.PREC_SPLIT, 2e-6)])
def test_autotune_and_step_graph(precision, tol):
    U = 13
    items, c, f = _batch(n=12, U=U, seed=4)
    plan = B.Plan(items, U, len(c), len(f), precision)
    cd = torch.as_tensor(c).cuda()
    fd = torch.as_tensor(f).cuda()
    co = cd.clone()
    chosen = plan.autotune(cd, fd, co)
    assert chosen == plan.tuning
    # the step graph replays interpolate + restrict on the captured buffers
    fd.copy_(torch.as_tensor(f))
    co.copy_(cd)
    plan.capture_step(cd, fd, co)
    for _ in range(2):
        plan.launch_step()
    torch.cuda.synchronize()
    _check(items, U, c, f, fd.cpu().numpy(), co.cpu().numpy(), tol)


def test_launch_without_capture_rejected():
    items, c, f = _batch(n=2)
    plan = B.Plan(items, 13, len(c), len(f))
    with pytest.raises(B.AmrError):
        plan.launch_step()
