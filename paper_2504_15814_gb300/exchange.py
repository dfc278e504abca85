"""Face-array exchange between ranks around the transfer.

In a distributed spacetree code the coarse patch of a hanging face and its
nine fine patches may live on different ranks (the paper's code exchanges
such data at MPI boundaries; Sec. 6).  The transfer of one item runs on the
rank that holds its fine face arrays (its ghost halves are written there);
the coarse face array it reads, and whose fine-side half it restricts into,
belongs to the coarse patch's rank.  One step then is:

  1. ``pull``: every rank receives a copy of each remote coarse face array
     its items read (the whole 2k p^2 U array: interpolation stencils reach
     into both halves);
  2. interpolate + restrict locally (one plan over local buffers);
  3. ``push``: every rank sends back the coarse halo volumes its items
     restricted into remote arrays -- only the volumes its subfaces own, so
     subfaces of one hanging face spread over several ranks merge without
     overlap -- and the owner scatters them into its array.

Both steps are point-to-point sends of gathered buffers through
``torch.distributed`` (NCCL for device tensors, gloo for host tensors); no
multicast and no collective.  The index lists are built once from the global
item list, identically on every rank, so message sizes always agree.
"""
import numpy as np

from .workloads import face_axes


def restricted_elements(item, U):
    """Element offsets, relative to the start of the item's coarse face array,
    of the coarse halo values the item's restriction writes: fine-side layers
    j = 0..k-1, tangential indices owned by its subfaces (coarse a is owned by
    the subface holding fine index 3a + 1)."""
    face, sub = int(item["face"]), int(item["subface"])
    p, k = int(item["patch_size"]), int(item["overlap"])
    n, t0, t1 = face_axes(face)
    ext = [p, p, p]
    ext[n] = 2 * k
    out = []
    for s in (range(9) if sub < 0 else [sub]):
        r0 = range((s % 3 * p + 1) // 3, (s % 3 * p + p + 1) // 3)
        r1 = range((s // 3 * p + 1) // 3, (s // 3 * p + p + 1) // 3)
        for j in range(k):
            for b in r1:
                for a in r0:
                    idx = [0, 0, 0]
                    idx[n] = k + j if face < 3 else k - 1 - j
                    idx[t0], idx[t1] = a, b
                    vol = (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]
                    out.append(vol * U + np.arange(U))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


class FaceExchange:
    """Local layout of one rank and the exchange lists of all ranks.

    items        global item list (workloads.ITEM_DTYPE) with offsets into a
                 virtual global coarse / fine buffer;
    coarse_owner mapping coarse_offset -> rank owning that coarse face array;
    fine_owner   per item, the rank holding its fine face arrays (the rank
                 that runs its transfer).

    Attributes of this rank: ``items`` (its transfer items on local
    buffers), ``coarse_len`` / ``fine_len`` (local buffer sizes: its own
    coarse arrays first, then copies of remote ones), ``coarse_src`` /
    ``fine_src`` ((global offset, local offset, length) of the arrays it
    owns, to lay out local buffers from global data)."""

    def __init__(self, items, U, coarse_owner, fine_owner, rank, world, align=2):
        self.rank, self.world, self.U = rank, world, U
        fine_owner = np.asarray(fine_owner)
        arr_len = {}
        for it in items:
            p, k = int(it["patch_size"]), int(it["overlap"])
            arr_len[int(it["coarse_offset"])] = 2 * k * p * p * U
        pad = lambda n: -(-n // align) * align
        # local coarse layout of every rank: owned arrays, then remote copies
        layouts = []
        for r in range(world):
            loc, off = {}, 0
            for g in sorted(arr_len):
                if coarse_owner[g] == r:
                    loc[g] = off
                    off += pad(arr_len[g])
            for i in np.flatnonzero(fine_owner == r):
                g = int(items[i]["coarse_offset"])
                if g not in loc:
                    loc[g] = off
                    off += pad(arr_len[g])
            layouts.append((loc, off))
        loc, self.coarse_len = layouts[rank]
        self.coarse_src = [(g, loc[g], arr_len[g]) for g in sorted(arr_len) if coarse_owner[g] == rank]
        # local fine layout and items of this rank
        mine = np.flatnonzero(fine_owner == rank)
        self.item_index = mine
        self.items = items[mine].copy()
        self.fine_src, fo = [], 0
        for q, i in enumerate(mine):
            it = items[i]
            nf = (9 if int(it["subface"]) < 0 else 1) * arr_len[int(it["coarse_offset"])]
            self.fine_src.append((int(it["fine_offset"]), fo, nf))
            self.items[q]["coarse_offset"] = loc[int(it["coarse_offset"])]
            self.items[q]["fine_offset"] = fo
            fo += pad(nf)
        self.fine_len = fo
        # pull: owner -> reader, whole arrays, once per (array, reader rank)
        self.pull_send = {r: [] for r in range(world)}
        self.pull_recv = {r: [] for r in range(world)}
        # push: reader -> owner, owned halo elements of the reader's items
        self.push_send = {r: [] for r in range(world)}
        self.push_recv = {r: [] for r in range(world)}
        for reader in range(world):
            rloc = layouts[reader][0]
            seen = set()
            for i in np.flatnonzero(fine_owner == reader):
                g = int(items[i]["coarse_offset"])
                owner = coarse_owner[g]
                if owner == reader:
                    continue
                oloc = layouts[owner][0]
                if g not in seen:
                    seen.add(g)
                    whole = np.arange(arr_len[g], dtype=np.int64)
                    if owner == rank:
                        self.pull_send[reader].append(oloc[g] + whole)
                    if reader == rank:
                        self.pull_recv[owner].append(rloc[g] + whole)
                el = restricted_elements(items[i], U)
                if reader == rank:
                    self.push_send[owner].append(rloc[g] + el)
                if owner == rank:
                    self.push_recv[reader].append(oloc[g] + el)
        cat = lambda v: np.concatenate(v) if v else np.zeros(0, dtype=np.int64)
        for d in (self.pull_send, self.pull_recv, self.push_send, self.push_recv):
            for r in d:
                d[r] = cat(d[r])
        self._idx = {}

    def _index(self, key, arr, device):
        k = (key, str(device))
        if k not in self._idx:
            import torch
            self._idx[k] = torch.as_tensor(arr, dtype=torch.int64, device=device)
        return self._idx[k]

    def _exchange(self, buf, send, recv, tag):
        import torch
        import torch.distributed as dist
        ops, pending = [], []
        for peer in range(self.world):
            if peer == self.rank:
                continue
            if len(send[peer]):
                sbuf = buf[self._index((tag, "s", peer), send[peer], buf.device)]
                ops.append(dist.P2POp(dist.isend, sbuf, peer))
            if len(recv[peer]):
                rbuf = torch.empty(len(recv[peer]), dtype=buf.dtype, device=buf.device)
                ops.append(dist.P2POp(dist.irecv, rbuf, peer))
                pending.append((peer, rbuf))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        for peer, rbuf in pending:
            buf[self._index((tag, "r", peer), recv[peer], buf.device)] = rbuf

    def pull(self, coarse_local):
        """Receive copies of the remote coarse face arrays this rank's items
        read (and send this rank's arrays to their readers)."""
        self._exchange(coarse_local, self.pull_send, self.pull_recv, "pull")

    def push(self, coarse_local):
        """Send the coarse halo volumes this rank restricted into copies of
        remote arrays to their owners (and scatter the ones received)."""
        self._exchange(coarse_local, self.push_send, self.push_recv, "push")

    def bytes_per_step(self):
        """Bytes this rank sends per step (pull + push), float64 values."""
        n = sum(len(v) for v in self.pull_send.values()) + sum(len(v) for v in self.push_send.values())
        return 8 * n
