"""Multi-GPU sharding logic on CPU ranks (gloo, world size 2): the shards
cover every item once, are cost balanced, and the union of the per-rank
results (the oracle standing in for each rank's GPU) equals the single-rank
result -- so the data path needs no collective."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import transfer as tr
from paper_2504_15814_gb300 import sharding as S
from paper_2504_15814_gb300 import workloads as wl


def test_bounds_cover_and_balance():
    items, _, _ = wl.make_items([0] * 10 + [1] * 7, [-1] * 10 + [3] * 7, [9] * 10 + [6] * 7, [3] * 17,
                                [3] * 5 + [1] * 12, 4)
    for world in (1, 2, 3, 5, 40):
        b = S.shard_bounds(items, world)
        assert b[0][0] == 0 and b[-1][1] == len(items)
        assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
        assert all(lo <= hi for lo, hi in b)
    cost = S.item_cost(items)
    b = S.shard_bounds(items, 2)
    c0, c1 = cost[b[0][0]:b[0][1]].sum(), cost[b[1][0]:b[1][1]].sum()
    assert abs(c0 - c1) <= cost.max()


def test_items_sharing_a_coarse_array_stay_on_one_rank():
    """Subface items of one hanging face listed separately (and interleaved
    with other items) name the same coarse array; no shard boundary may
    separate them, whatever the world size."""
    U = 2
    faces = [0, 1, 0, 2, 0, 3, 1, 4, 5, 0]
    subs = [0, 0, 4, 0, 8, 0, 5, 0, 0, 2]
    items, cl, fl = wl.make_items(faces, subs, [6] * 10, [2] * 10, [3] * 10, U)
    arr = 2 * 2 * 36 * U
    # items 0, 2, 4, 9 share face 0's coarse array; items 1 and 6 share face 1's
    shared = {0: 0, 2: 0, 4: 0, 9: 0, 1: 1, 6: 1}
    for i, grp in shared.items():
        items[i]["coarse_offset"] = cl + grp * arr  # past the private arrays: no accidental sharing
    ok = S.allowed_cuts(items)
    assert ok[0] and ok[10] and not ok[1:10].any()
    for world in (2, 3, 4):
        for lo, hi in S.shard_bounds(items, world):
            for grp in (0, 1):
                members = [i for i, g in shared.items() if g == grp]
                inside = [lo <= i < hi for i in members]
                assert all(inside) or not any(inside)
    # contiguous runs: a cut is allowed between the groups
    items2 = items[[0, 2, 4, 9, 1, 6, 3, 5, 7, 8]]
    ok2 = S.allowed_cuts(items2)
    assert list(np.flatnonzero(ok2)) == [0, 4, 6, 7, 8, 9, 10]
    b = S.shard_bounds(items2, 2)
    assert b[0][1] in (4, 6, 7, 8, 9)


def test_local_items_share_coarse_arrays():
    U = 3
    arr = 2 * 2 * 36 * U
    items = np.zeros(3, dtype=wl.ITEM_DTYPE)
    for s in range(3):
        items[s] = (4, s, 6, 2, 2, 0, 5 * arr, 100 + s * arr)
    sub, cl, fl, csrc, fsrc = S.local_items(items, U, 0, 3)
    assert len(csrc) == 1 and cl >= arr
    assert set(sub["coarse_offset"]) == {0}
    assert [f[0] for f in fsrc] == [100, 100 + arr, 100 + 2 * arr]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shared_batch(U):
    """Subface items of three hanging faces listed separately and interleaved
    with private items: every hanging face's subface items name one coarse
    array."""
    n = 16
    faces = [0, 1, 0, 2, 1, 0, 3, 2, 1, 4, 2, 5, 0, 1, 2, 3]
    subs = [0, 3, 4, 1, 5, 8, 2, 4, 7, 6, 8, 0, 2, 1, 6, 7]
    items, cl, fl = wl.make_items(faces, subs, [6] * n, [3] * n, [3, 2, 1, 3] * 4, U)
    arr = 2 * 3 * 36 * U
    groups = {0: [0, 2, 5, 12], 1: [1, 4, 8, 13], 2: [3, 7, 10, 14]}
    for g, members in groups.items():
        for i in members:
            items[i]["coarse_offset"] = cl + g * arr
    cl += 3 * arr
    rng = np.random.Generator(np.random.PCG64(wl.SEED_BASE + 900))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(n, rng))
    return items, coarse, fine


def _rank_main(rank, world, port, U, out_dir, shared=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if shared:
        items, coarse, fine = _shared_batch(U)
    else:
        items, coarse, fine = wl.uneven_batch(n_items=24, U=U, config_index=2)
    c, f = coarse.numpy(), fine.numpy()
    lo, hi = S.shard_bounds(items, world)[rank]
    sub, cl, fl, csrc, fsrc = S.local_items(items, U, lo, hi)
    lc, lf = np.zeros(cl), np.zeros(fl)
    for g, l, n in csrc:
        lc[l:l + n] = c[g:g + n]
    for g, l, n in fsrc:
        lf[l:l + n] = f[g:g + n]
    # each rank runs its own shard (the oracle stands in for its GPU)
    lf_out = tr.interpolate(sub, U, lc, lf)
    lc_out = tr.restrict(sub, U, lf_out, lc)
    # scatter back into global buffers and combine only to verify the result
    gf = torch.zeros(len(f), dtype=torch.float64)
    gc = torch.zeros(len(c), dtype=torch.float64)
    mf = torch.zeros(len(f), dtype=torch.float64)
    mc = torch.zeros(len(c), dtype=torch.float64)
    for g, l, n in fsrc:
        gf[g:g + n] = torch.from_numpy(lf_out[l:l + n])
        mf[g:g + n] = 1
    for g, l, n in csrc:
        gc[g:g + n] = torch.from_numpy(lc_out[l:l + n])
        mc[g:g + n] = 1
    for t in (gf, gc, mf, mc):
        dist.all_reduce(t)
    if rank == 0:
        ref_f = tr.interpolate(items, U, c, f)
        ref_c = tr.restrict(items, U, ref_f, c)
        np.save(os.path.join(out_dir, "result.npy"),
                np.array([float(np.abs(gf.numpy() - ref_f)[mf.numpy() > 0].max()),
                          float(np.abs(gc.numpy() - ref_c)[mc.numpy() > 0].max()),
                          float(mf.max()), float(mc.max())]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("shared", [False, True])
def test_two_rank_shards_reproduce_single_rank(tmp_path, shared):
    U = 5
    mp.spawn(_rank_main, args=(2, _free_port(), U, str(tmp_path), shared), nprocs=2, join=True)
    ef, ec, mf, mc = np.load(tmp_path / "result.npy")
    assert ef == 0.0 and ec == 0.0   # bit-identical: same operators, same data
    assert mf == 1.0 and mc == 1.0   # every array owned by exactly one rank
