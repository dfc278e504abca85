"""Seeded synthetic transfer workloads: item lists and face-array buffers.

This module only lays out buffers and samples smooth fields at cell centres;
it contains no interpolation or restriction arithmetic.  Tests feed the same
buffers to the CUDA path and to the CPU oracle, and ``bench.py`` times the
CUDA path on them.

Layout convention (shared by every part of the library):
  face f: normal axis n = f % 3, tangential axes t0 < t1; f < 3 puts the
  coarse patch on the low side of the interface, f >= 3 on the high side.
  Face array: extent 2k along n, p along t0 and t1, lexicographic with x
  fastest, U unknowns per volume innermost (AoS), float64.
  Normal index i sits at (i - k + 1/2) * spacing from the interface.
  Coarse tangential index a sits at (a + 1/2) H; subface s = s0 + 3 s1's fine
  tangential index q sits at (s_t p + q + 1/2) H / 3.

Field recipes (units: one coarse cell H = 1; positions are item origin + the
face-frame position, the face frame being axis aligned):
  smooth     per unknown, 4 Gaussians (amplitude U[-1,1], width U[2,8] H,
             centre in the 64 H cube) + 4 plane sinusoids (amplitude U[-1,1],
             wavelength U[4,16] H, random unit direction, phase U[0, 2 pi]),
             plus 1e-8 * max|u| * U[-1,1] noise per element;
  puncture   per unknown u mod 3: (0) psi = 1 + M / (2 r), r = max(|x - x_p|,
             H/2), M ~ U[0.5, 1]; (1) a lapse-like field, the Gaussian-smoothed
             inverse square psi_s^-2 with psi_s = 1 + M / (2 sqrt(r^2 + w^2)),
             w ~ U[1,2] H; (2) shift-like Gaussian bumps (3 per unknown,
             amplitude U[-0.5,0.5], width U[1,4] H); x_p within 3 H of the
             face plane of each item;
  polynomial a callable f(xyz) -> (N, U) evaluated at cell centres.
"""
import math

import numpy as np
import torch

ITEM_DTYPE = np.dtype([
    ("face", "<i4"), ("subface", "<i4"), ("patch_size", "<i4"), ("overlap", "<i4"),
    ("order", "<i4"), ("scheme", "<i4"), ("coarse_offset", "<i8"), ("fine_offset", "<i8"),
])

SEED_BASE = 2504_15814


def face_axes(face):
    n = face % 3
    t0, t1 = [d for d in range(3) if d != n]
    return n, t0, t1


def array_volumes(p, k):
    return 2 * k * p * p


def make_items(faces, subfaces, ps, ks, orders, U, align=2):
    """Items with private, consecutively packed coarse and fine face arrays.

    faces/subfaces/ps/ks/orders: equal-length integer sequences.  A whole-face
    item (subface -1) owns nine fine arrays.  Each array starts on a multiple
    of ``align`` elements.  Returns (items, coarse_len, fine_len)."""
    n = len(faces)
    items = np.zeros(n, dtype=ITEM_DTYPE)
    co = fo = 0
    for i in range(n):
        p, k = int(ps[i]), int(ks[i])
        vol = array_volumes(p, k) * U
        nsub = 9 if int(subfaces[i]) < 0 else 1
        items[i] = (int(faces[i]), int(subfaces[i]), p, k, int(orders[i]), 0, co, fo)
        co += -(-vol // align) * align
        fo += -(-(nsub * vol) // align) * align
    return items, co, fo


def volume_positions(items, U, origins, device="cpu"):
    """Physical centres of every volume of every coarse and fine face array.

    Returns (coarse_pos, coarse_index, fine_pos, fine_index): positions (N, 3)
    float64 and the element offset of each volume's first unknown."""
    cpos, cidx, fpos, fidx = [], [], [], []
    for it, org in zip(items, origins):
        face, sub, p, k = int(it["face"]), int(it["subface"]), int(it["patch_size"]), int(it["overlap"])
        n, t0, t1 = face_axes(face)
        ext = [p, p, p]
        ext[n] = 2 * k
        iz, iy, ix = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]), indexing="ij")
        idx = [ix.ravel(), iy.ravel(), iz.ravel()]
        nvol = idx[0].size
        vol_elems = nvol * U
        # coarse array
        x = np.zeros((nvol, 3))
        x[:, n] = idx[n] - k + 0.5
        x[:, t0] = idx[t0] + 0.5
        x[:, t1] = idx[t1] + 0.5
        cpos.append(x + org)
        cidx.append(int(it["coarse_offset"]) + np.arange(nvol) * U)
        subs = [(j, j) for j in range(9)] if sub < 0 else [(sub, 0)]
        for s, j in subs:
            s0, s1 = s % 3, s // 3
            x = np.zeros((nvol, 3))
            x[:, n] = (idx[n] - k + 0.5) / 3.0
            x[:, t0] = (s0 * p + idx[t0] + 0.5) / 3.0
            x[:, t1] = (s1 * p + idx[t1] + 0.5) / 3.0
            fpos.append(x + org)
            fidx.append(int(it["fine_offset"]) + j * vol_elems + np.arange(nvol) * U)
    cat = lambda a, dt: torch.from_numpy(np.concatenate(a).astype(dt)).to(device)
    return cat(cpos, np.float64), cat(cidx, np.int64), cat(fpos, np.float64), cat(fidx, np.int64)


def _scatter(buf, start_idx, values, U):
    """buf[start_idx[v] + u] = values[v, u]."""
    cols = start_idx[:, None] + torch.arange(U, device=buf.device)[None, :]
    buf[cols.reshape(-1)] = values.reshape(-1)


def sample_buffers(items, U, coarse_len, fine_len, field, origins, device="cpu", chunk=1 << 18):
    """Fill fresh coarse and fine buffers (float64 on ``device``) with
    field(positions (N,3) float64 tensor) -> (N, U) tensor at every volume."""
    cpos, cidx, fpos, fidx = volume_positions(items, U, origins, device)
    coarse = torch.zeros(coarse_len, dtype=torch.float64, device=device)
    fine = torch.zeros(fine_len, dtype=torch.float64, device=device)
    for buf, pos, idx in ((coarse, cpos, cidx), (fine, fpos, fidx)):
        for s in range(0, pos.shape[0], chunk):
            _scatter(buf, idx[s:s + chunk], field(pos[s:s + chunk]), U)
    return coarse, fine


class SmoothField:
    """Sum of 4 Gaussians and 4 sinusoids per unknown (see module docstring)."""

    def __init__(self, U, rng, box=64.0, device="cpu"):
        f = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)
        self.g_amp = f(rng.uniform(-1, 1, (U, 4)))
        self.g_w = f(rng.uniform(2, 8, (U, 4)))
        self.g_c = f(rng.uniform(0, box, (U, 4, 3)))
        self.s_amp = f(rng.uniform(-1, 1, (U, 4)))
        lam = rng.uniform(4, 16, (U, 4))
        d = rng.normal(size=(U, 4, 3))
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        self.s_k = f(d * (2 * math.pi / lam)[..., None])
        self.s_ph = f(rng.uniform(0, 2 * math.pi, (U, 4)))

    def __call__(self, x):
        r2 = ((x[:, None, None, :] - self.g_c[None]) ** 2).sum(-1)           # (N, U, 4)
        v = (self.g_amp * torch.exp(-r2 / self.g_w ** 2)).sum(-1)
        ph = (x[:, None, None, :] * self.s_k[None]).sum(-1) + self.s_ph       # (N, U, 4)
        return v + (self.s_amp * torch.sin(ph)).sum(-1)


class PunctureField:
    """Puncture-like profiles (see module docstring); one puncture per item."""

    def __init__(self, U, rng, punctures, device="cpu"):
        f = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)
        self.U = U
        self.M = f(rng.uniform(0.5, 1.0, U))
        self.w = f(rng.uniform(1.0, 2.0, U))
        self.b_amp = f(rng.uniform(-0.5, 0.5, (U, 3)))
        self.b_w = f(rng.uniform(1.0, 4.0, (U, 3)))
        self.b_off = f(rng.uniform(-3.0, 3.0, (U, 3, 3)))
        self.punctures = punctures  # (N, 3) per-volume puncture position, set by the caller

    def __call__(self, x, xp):
        r2 = ((x - xp) ** 2).sum(-1, keepdim=True)                          # (N, 1)
        r = torch.sqrt(r2).clamp_min(0.5)
        psi = 1.0 + self.M[None] / (2.0 * r)
        psi_s = 1.0 + self.M[None] / (2.0 * torch.sqrt(r2 + self.w[None] ** 2))
        lapse = psi_s ** -2
        c = xp[:, None, None, :] + self.b_off[None]
        bump = (self.b_amp * torch.exp(-((x[:, None, None, :] - c) ** 2).sum(-1) / self.b_w ** 2)).sum(-1)
        kind = torch.arange(self.U, device=x.device) % 3
        return torch.where(kind == 0, psi, torch.where(kind == 1, lapse, bump))


def add_noise(buf, rel, rng):
    """buf += rel * max|buf| * U[-1,1] (seeded, generated on the host)."""
    if rel == 0 or buf.numel() == 0:
        return buf
    scale = rel * float(buf.abs().max())
    g = torch.Generator(device="cpu").manual_seed(int(rng.integers(1 << 62)))
    buf += ((torch.rand(buf.numel(), generator=g, dtype=torch.float64) * 2 - 1) * scale).to(buf.device)
    return buf


def origins_in_box(n, rng, box=64.0):
    return rng.uniform(0, box, (n, 3))


def uniform_batch(n_faces=2048, p=9, k=3, U=59, order=3, config_index=1, device="cpu",
                  noise=1e-8, faces=None, shard=None):
    """Hanging faces as whole-face items (nine subfaces each), faces cycled
    0..5, smooth fields.  shard=(rank, world) keeps only that rank's
    cost-balanced share of the n_faces items, on compact local buffers.
    Returns (items, coarse, fine)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + config_index))
    if faces is None:
        faces = [i % 6 for i in range(n_faces)]
    items, cl, fl = make_items(faces, [-1] * n_faces, [p] * n_faces, [k] * n_faces,
                               [order] * n_faces, U)
    origins = origins_in_box(n_faces, rng)
    field = SmoothField(U, rng, device=device)
    if shard is not None:
        from .sharding import local_items, shard_bounds
        rank, world = shard
        lo, hi = shard_bounds(items, world)[rank]
        items, cl, fl, _, _ = local_items(items, U, lo, hi)
        origins = origins[lo:hi]
    coarse, fine = sample_buffers(items, U, cl, fl, field, origins, device)
    add_noise(coarse, noise, rng)
    add_noise(fine, noise, rng)
    return items, coarse, fine


def uneven_batch(n_items=20000, U=59, config_index=2, device="cpu", noise=1e-8):
    """Single-subface items with p in {6, 9, 12} (40/40/20 %), k in {2, 3},
    order in {1, 2, 3}, random face and subface, smooth fields."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + config_index))
    ps = rng.choice([6, 9, 12], size=n_items, p=[0.4, 0.4, 0.2])
    ks = rng.choice([2, 3], size=n_items)
    orders = rng.choice([1, 2, 3], size=n_items)
    faces = rng.integers(0, 6, n_items)
    subs = rng.integers(0, 9, n_items)
    items, cl, fl = make_items(faces, subs, ps, ks, orders, U)
    origins = origins_in_box(n_items, rng)
    field = SmoothField(U, rng, device=device)
    coarse, fine = sample_buffers(items, U, cl, fl, field, origins, device)
    add_noise(coarse, noise, rng)
    add_noise(fine, noise, rng)
    return items, coarse, fine


def puncture_batch(n_faces=8192, p=9, k=3, U=59, order=3, config_index=3, device="cpu"):
    """Hanging faces with puncture-like fields; each item's puncture lies
    within 3 H of its face plane, over the face."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + config_index))
    faces = [i % 6 for i in range(n_faces)]
    items, cl, fl = make_items(faces, [-1] * n_faces, [p] * n_faces, [k] * n_faces,
                               [order] * n_faces, U)
    origins = origins_in_box(n_faces, rng)
    pf = PunctureField(U, rng, None, device=device)
    xp = np.zeros((n_faces, 3))
    for i, f in enumerate(faces):
        n, t0, t1 = face_axes(f)
        xp[i, n] = origins[i, n] + rng.uniform(-3, 3)
        xp[i, t0] = origins[i, t0] + rng.uniform(0, p)
        xp[i, t1] = origins[i, t1] + rng.uniform(0, p)
    cpos, cidx, fpos, fidx = volume_positions(items, U, origins, device)
    per_item_c = np.repeat(np.arange(n_faces), [array_volumes(p, k)] * n_faces)
    per_item_f = np.repeat(np.arange(n_faces), [9 * array_volumes(p, k)] * n_faces)
    xp_t = torch.as_tensor(xp, dtype=torch.float64, device=device)
    coarse = torch.zeros(cl, dtype=torch.float64, device=device)
    fine = torch.zeros(fl, dtype=torch.float64, device=device)
    chunk = 1 << 18
    for buf, pos, idx, owner in ((coarse, cpos, cidx, per_item_c), (fine, fpos, fidx, per_item_f)):
        own = torch.as_tensor(owner, device=device)
        for s in range(0, pos.shape[0], chunk):
            _scatter(buf, idx[s:s + chunk], pf(pos[s:s + chunk], xp_t[own[s:s + chunk]]), U)
    return items, coarse, fine


def polynomial_buffers(items, U, coarse_len, fine_len, poly, origins=None, device="cpu"):
    """Buffers sampled from poly(xyz (N,3)) -> (N, U) at every volume."""
    if origins is None:
        origins = np.zeros((len(items), 3))
    return sample_buffers(items, U, coarse_len, fine_len, poly, origins, device)
