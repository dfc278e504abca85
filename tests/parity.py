"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare them per (item, unknown)."""
import json
import os

import numpy as np
import torch

from oracle import transfer as tr


def item_slices(items, U):
    """Per item: ((coarse lo, hi), (fine lo, hi)) element ranges of its arrays."""
    out = []
    for it in items:
        p, k = int(it["patch_size"]), int(it["overlap"])
        arr = 2 * k * p * p * U
        nsub = 9 if int(it["subface"]) < 0 else 1
        co, fo = int(it["coarse_offset"]), int(it["fine_offset"])
        out.append(((co, co + arr), (fo, fo + nsub * arr)))
    return out


def written_masks(items, U, cl, fl):
    """Boolean masks of the fine entries interpolate writes and the coarse
    entries restrict writes (found by running the oracle on NaN buffers)."""
    f = tr.interpolate(items, U, np.zeros(cl), np.full(fl, np.nan))
    c = tr.restrict(items, U, np.zeros(fl), np.full(cl, np.nan))
    return ~np.isnan(f), ~np.isnan(c)


def normwise_errors(items, U, got, ref, mask, which):
    """Max over items and unknowns of max|got - ref| / max|ref| over the
    written entries of that item's arrays, and the RMS of the same ratios."""
    worst, ratios = 0.0, []
    for (c_rng, f_rng) in item_slices(items, U):
        lo, hi = f_rng if which == "fine" else c_rng
        g = got[lo:hi].reshape(-1, U)
        r = ref[lo:hi].reshape(-1, U)
        m = mask[lo:hi].reshape(-1, U)
        for u in range(U):
            sel = m[:, u]
            if not sel.any():
                continue
            err = np.abs(g[sel, u] - r[sel, u]).max()
            scale = max(np.abs(r[sel, u]).max(), 1e-300)
            ratios.append(err / scale)
            worst = max(worst, err / scale)
    rms = float(np.sqrt(np.mean(np.square(ratios)))) if ratios else 0.0
    return worst, rms


def gpu_interpolate(plan, coarse, fine):
    c = torch.as_tensor(coarse).cuda()
    f = torch.as_tensor(fine).cuda().clone()
    plan.interpolate(c, f)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def gpu_restrict(plan, fine, coarse):
    f = torch.as_tensor(fine).cuda()
    c = torch.as_tensor(coarse).cuda().clone()
    plan.restrict(f, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def record(**kw):
    """Append measured errors to $AMR_PARITY_LOG (JSON lines) when it is set."""
    path = os.environ.get("AMR_PARITY_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(kw) + "\n")
