"""Splitting a transfer item list across GPUs.

Transfer items are independent (every hanging face or subface reads its own
coarse and fine face arrays and writes its own outputs), except that items
naming the same coarse face array (subfaces of one hanging face) restrict
into that one array and must stay together.  N GPUs each take a contiguous,
cost-balanced range of the items that keeps such items together and run
their own plan on local buffers: no collective is needed on the data path
(weak scaling when every GPU keeps the same amount of work).  When the coarse
and fine sides of a face live on different ranks, ``exchange`` moves the
face arrays between them around the transfer.
"""
import numpy as np


def item_cost(items):
    """Relative cost of each item: written volumes (k p^2 per subface) times
    the order's stencil weight (d-linear 1, Taylor-2 2, Taylor-3 3)."""
    nsub = np.where(items["subface"] < 0, 9, 1)
    return nsub * items["overlap"].astype(np.int64) * items["patch_size"].astype(np.int64) ** 2 * items["order"]


def allowed_cuts(items):
    """Boolean array over cut positions 0..n: a cut at position c (ranks take
    items [.., c) and [c, ..)) is allowed when no two items that share a
    coarse face array lie on different sides of it.  Such items (subfaces of
    one hanging face, listed separately) all restrict into the same coarse
    array, so they must run on the same rank."""
    n = len(items)
    ok = np.ones(n + 1, dtype=bool)
    if n == 0:
        return ok
    co = np.asarray(items["coarse_offset"], dtype=np.int64)
    order = np.argsort(co, kind="stable")
    sco = co[order]
    starts = np.flatnonzero(np.concatenate([[True], sco[1:] != sco[:-1]]))
    ends = np.concatenate([starts[1:], [n]])
    for a, b in zip(starts, ends):
        if b - a > 1:
            members = order[a:b]
            ok[members.min() + 1:members.max() + 1] = False
    return ok


def shard_bounds(items, world):
    """[lo_r, hi_r) item ranges of the world ranks, contiguous, balanced by
    item_cost, covering every item exactly once (ranks may be empty), never
    separating items that share a coarse face array (see allowed_cuts)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    prefix = np.concatenate([[0], np.cumsum(item_cost(items))]) if len(items) else np.zeros(1, dtype=np.int64)
    total = int(prefix[-1])
    ok = allowed_cuts(items)
    cand = np.flatnonzero(ok)
    bounds = [0]
    for r in range(1, world):
        # the allowed cut whose prefix cost is closest to r/world of the total
        n = int(cand[np.argmin(np.abs(prefix[cand] - total * r / world))])
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
