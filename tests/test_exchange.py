"""Face-array exchange between ranks (gloo, world size 2, CPU tensors).

A global batch whose coarse face arrays and fine face arrays are owned by
different ranks -- including one hanging face whose nine subfaces run on both
ranks -- is transferred per rank as pull, interpolate + restrict (the oracle
stands in for each rank's GPU), push.  The union of the per-rank results must
equal the single-rank result bit for bit: every ghost half, and every coarse
halo volume written back to its owner."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import transfer as tr
from paper_2504_15814_gb300 import exchange as X
from paper_2504_15814_gb300 import workloads as wl


def _problem(U):
    # items 0..8: the nine subfaces of one hanging face (face 1), sharing a
    # coarse array; items 9..14: whole faces and subfaces with private arrays
    faces = [1] * 9 + [0, 2, 3, 4, 5, 0]
    subs = list(range(9)) + [-1, 4, -1, 0, 8, -1]
    n = len(faces)
    items, cl, fl = wl.make_items(faces, subs, [6] * n, [3] * n, [3, 2, 1] * 5, U)
    arr = 2 * 3 * 36 * U
    items[:9]["coarse_offset"] = cl
    cl += arr
    rng = np.random.Generator(np.random.PCG64(wl.SEED_BASE + 901))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(n, rng))
    groups = sorted({int(o) for o in items["coarse_offset"]})
    coarse_owner = {g: (q % 2) for q, g in enumerate(groups)}
    coarse_owner[cl - arr] = 0  # the shared array lives on rank 0
    fine_owner = np.array([0, 1, 1, 0, 1, 0, 1, 1, 0, 1, 0, 0, 1, 1, 0])
    return items, coarse.numpy(), fine.numpy(), coarse_owner, fine_owner


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, U, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items, c, f, coarse_owner, fine_owner = _problem(U)
    ex = X.FaceExchange(items, U, coarse_owner, fine_owner, rank, world)
    lc = torch.zeros(ex.coarse_len, dtype=torch.float64)
    lf = torch.zeros(ex.fine_len, dtype=torch.float64)
    for g, l, n in ex.coarse_src:
        lc[l:l + n] = torch.from_numpy(c[g:g + n])
    for g, l, n in ex.fine_src:
        lf[l:l + n] = torch.from_numpy(f[g:g + n])
    ex.pull(lc)
    lf_out = torch.from_numpy(tr.interpolate(ex.items, U, lc.numpy(), lf.numpy()))
    lc_out = torch.from_numpy(tr.restrict(ex.items, U, lf_out.numpy(), lc.numpy()))
    ex.push(lc_out)
    # collect the owned arrays of every rank into global buffers to compare
    gf, mf = torch.zeros(len(f), dtype=torch.float64), torch.zeros(len(f), dtype=torch.float64)
    gc, mc = torch.zeros(len(c), dtype=torch.float64), torch.zeros(len(c), dtype=torch.float64)
    for g, l, n in ex.fine_src:
        gf[g:g + n] = lf_out[l:l + n]
        mf[g:g + n] = 1
    for g, l, n in ex.coarse_src:
        gc[g:g + n] = lc_out[l:l + n]
        mc[g:g + n] = 1
    for t in (gf, gc, mf, mc):
        dist.all_reduce(t)
    sent = torch.tensor([float(ex.bytes_per_step())])
    dist.all_reduce(sent)
    if rank == 0:
        ref_f = tr.interpolate(items, U, c, f)
        ref_c = tr.restrict(items, U, ref_f, c)
        np.save(os.path.join(out_dir, "result.npy"),
                np.array([float(np.abs(gf.numpy() - ref_f)[mf.numpy() > 0].max()),
                          float(np.abs(gc.numpy() - ref_c)[mc.numpy() > 0].max()),
                          float(mf.max()), float(mc.max()), float(mf.min()), float(sent.item())]))
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_reproduces_single_rank(tmp_path):
    U = 3
    mp.spawn(_rank_main, args=(2, _free_port(), U, str(tmp_path)), nprocs=2, join=True)
    ef, ec, mf_max, mc_max, mf_min, sent = np.load(tmp_path / "result.npy")
    assert ef == 0.0 and ec == 0.0
    assert mf_max == 1.0 and mc_max == 1.0 and mf_min == 1.0  # every array owned exactly once
    assert sent > 0  # something crossed ranks


def test_restricted_elements_partition_the_halo():
    """The owned halo volumes of the nine subfaces tile the fine-side half of
    the coarse array exactly once (p a multiple of 3 or not)."""
    U = 2
    for p in (6, 7, 9):
        for face in range(6):
            k = 3
            items, _, _ = wl.make_items([face] * 9, list(range(9)), [p] * 9, [k] * 9, [3] * 9, U)
            els = np.concatenate([X.restricted_elements(it, U) for it in items])
            assert len(els) == len(set(els.tolist())) == k * p * p * U
            whole, _, _ = wl.make_items([face], [-1], [p], [k], [3], U)
            assert sorted(els.tolist()) == sorted(X.restricted_elements(whole[0], U).tolist())


def test_restricted_elements_are_what_restriction_writes():
    """The exchange sends back exactly the coarse entries the oracle's
    restriction writes for each item."""
    U = 2
    items, cl, fl = wl.make_items([0, 4, 2, 5], [3, -1, 8, 0], [7, 6, 9, 5], [2, 3, 3, 2], [3, 1, 2, 3], U)
    out = tr.restrict(items, U, np.zeros(fl), np.full(cl, np.nan))
    for it in items:
        co = int(it["coarse_offset"])
        arr = 2 * int(it["overlap"]) * int(it["patch_size"]) ** 2 * U
        written = np.flatnonzero(~np.isnan(out[co:co + arr]))
        assert sorted(X.restricted_elements(it, U).tolist()) == written.tolist()
