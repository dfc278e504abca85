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


def _rank_main(rank, world, port, U, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
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


def test_two_rank_shards_reproduce_single_rank(tmp_path):
    U = 5
    mp.spawn(_rank_main, args=(2, _free_port(), U, str(tmp_path)), nprocs=2, join=True)
    ef, ec, mf, mc = np.load(tmp_path / "result.npy")
    assert ef == 0.0 and ec == 0.0   # bit-identical: same operators, same data
    assert mf == 1.0 and mc == 1.0   # every array owned by exactly one rank
