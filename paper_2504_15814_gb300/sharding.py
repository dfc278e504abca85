"""Splitting a transfer item list across GPUs.

Transfer items are independent (every hanging face or subface reads its own
coarse and fine face arrays and writes its own outputs), so N GPUs each take a
contiguous, cost-balanced range of the items and run their own plan on local
buffers: no collective is needed on the data path (weak scaling when every
GPU keeps the same amount of work).
"""
import numpy as np


def item_cost(items):
    """Relative cost of each item: written volumes (k p^2 per subface) times
    the order's stencil weight (d-linear 1, Taylor-2 2, Taylor-3 3)."""
    nsub = np.where(items["subface"] < 0, 9, 1)
    return nsub * items["overlap"].astype(np.int64) * items["patch_size"].astype(np.int64) ** 2 * items["order"]


def shard_bounds(items, world):
    """[lo_r, hi_r) item ranges of the world ranks, contiguous, balanced by
    item_cost, covering every item exactly once (ranks may be empty)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    prefix = np.concatenate([[0], np.cumsum(item_cost(items))]) if len(items) else np.zeros(1, dtype=np.int64)
    total = int(prefix[-1])
    bounds = [0]
    for r in range(1, world):
        # the prefix whose cost is closest to r/world of the total
        n = int(np.argmin(np.abs(prefix - total * r / world)))
        bounds.append(min(max(n, bounds[-1]), len(items)))
    bounds.append(len(items))
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def local_items(items, U, lo, hi, align=2):
    """Items [lo, hi) rebased onto compact local buffers.

    Returns (local_items, coarse_len, fine_len, coarse_src, fine_src) where
    coarse_src / fine_src list (global_offset, local_offset, length) copies
    that move each item's face arrays from the global layout to the local
    one.  Items that shared a coarse array globally share it locally."""
    sub = items[lo:hi].copy()
    coarse_map, coarse_src, fine_src = {}, [], []
    co = fo = 0
    for i in range(len(sub)):
        p, k = int(sub[i]["patch_size"]), int(sub[i]["overlap"])
        arr = 2 * k * p * p * U
        g_co = int(sub[i]["coarse_offset"])
        if g_co not in coarse_map:
            coarse_map[g_co] = co
            coarse_src.append((g_co, co, arr))
            co += -(-arr // align) * align
        nf = (9 if int(sub[i]["subface"]) < 0 else 1) * arr
        fine_src.append((int(sub[i]["fine_offset"]), fo, nf))
        sub[i]["coarse_offset"] = coarse_map[g_co]
        sub[i]["fine_offset"] = fo
        fo += -(-nf // align) * align
    return sub, co, fo, coarse_src, fine_src
