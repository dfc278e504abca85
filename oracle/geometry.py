"""Face-array layout and physical cell centres (paper Sec. 2).

A hanging face separates one coarse patch (p^3 volumes of width H) from the
3 x 3 fine patches (p^3 volumes of width h = H/3 each) that cover it
(three-partitioning, Sec. 2).  Data cross it as face arrays: 2k layers along
the face normal (k on each side, the halo depth) times p x p volumes
tangentially, all U unknowns of a volume stored together (AoS), volumes in
lexicographic order with x fastest (Sec. 4.1).

Conventions used throughout this repository:

* face f in 0..5 has normal axis n = f % 3; the tangential axes t0 < t1 are
  the other two in ascending order.  For f < 3 the coarse patch lies on the
  low side of the interface (negative normal coordinate), for f >= 3 on the
  high side.
* In a face array, normal index i_n in [0, 2k) sits at normal coordinate
  (i_n - k + 1/2) * spacing, the interface being at 0; tangential index i_t
  of the coarse array sits at (i_t + 1/2) * H.
* Subface s = s0 + 3 s1 (s0 along t0, s1 along t1) is the fine patch whose
  tangential index i_t sits at (s_t * p + i_t + 1/2) * h.  Coarse cell a
  covers fine global indices 3a .. 3a+2 and its centre coincides with fine
  3a + 1; when p is not a multiple of 3 a subface boundary can cut a coarse
  cell, which then belongs to the subface holding 3a + 1.
* Coordinates here are in units of H, in the face's own frame (origin at the
  face corner on the interface plane).
"""
from fractions import Fraction


def axes(face):
    """(normal axis, first tangential axis, second tangential axis)."""
    if not 0 <= face < 6:
        raise ValueError(f"face {face} not in 0..5")
    n = face % 3
    t0, t1 = [d for d in range(3) if d != n]
    return n, t0, t1


def coarse_side(face):
    """Sign of the normal coordinate on the coarse patch's own side."""
    return -1 if face < 3 else 1


def extents(face, p, k):
    """(E_x, E_y, E_z) of a face array in volumes."""
    n = axes(face)[0]
    ext = [p, p, p]
    ext[n] = 2 * k
    return tuple(ext)


def flat(ext, idx):
    """Lexicographic volume index, x fastest."""
    return (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]


def all_indices(ext):
    """Every (ix, iy, iz) of a box, in flat (x fastest) order."""
    return [(ix, iy, iz) for iz in range(ext[2]) for iy in range(ext[1]) for ix in range(ext[0])]


def coarse_centre(face, p, k, idx):
    """Centre of coarse face-array volume idx, in units of H."""
    n = axes(face)[0]
    half = Fraction(1, 2)
    x = [Fraction(idx[d]) + half for d in range(3)]
    x[n] = Fraction(idx[n] - k) + half
    return tuple(x)


def subface_pos(face, sub):
    """(s0, s1) of subface sub = s0 + 3 s1, placed on the face's (t0, t1)."""
    if not 0 <= sub < 9:
        raise ValueError(f"subface {sub} not in 0..8")
    return sub % 3, sub // 3


def fine_centre(face, p, k, sub, idx):
    """Centre of a volume of subface sub's fine face array, in units of H."""
    n, t0, t1 = axes(face)
    s0, s1 = subface_pos(face, sub)
    half = Fraction(1, 2)
    x = [None, None, None]
    x[n] = (Fraction(idx[n] - k) + half) / 3
    x[t0] = (Fraction(s0 * p + idx[t0]) + half) / 3
    x[t1] = (Fraction(s1 * p + idx[t1]) + half) / 3
    return tuple(x)


def fine_ghost_indices(face, p, k):
    """Fine face-array volumes on the coarse side: written by interpolation."""
    n = axes(face)[0]
    side = coarse_side(face)
    ext = extents(face, p, k)
    return [idx for idx in all_indices(ext) if (idx[n] - k + Fraction(1, 2)) * side > 0]


def owner_subface_index(a, p):
    """Subface index (along one tangential axis) owning coarse cell a: the one
    holding the fine cell 3a + 1 that coincides with the coarse centre."""
    return (3 * a + 1) // p


def coarse_halo_indices(face, p, k, sub):
    """Coarse face-array volumes on the fine side whose centre coincides with
    a fine centre of subface sub: written by restriction from that subface."""
    n, t0, t1 = axes(face)
    side = coarse_side(face)
    s0, s1 = subface_pos(face, sub)
    ext = extents(face, p, k)
    out = []
    for idx in all_indices(ext):
        if (idx[n] - k + Fraction(1, 2)) * side > 0:
            continue
        if owner_subface_index(idx[t0], p) == s0 and owner_subface_index(idx[t1], p) == s1:
            out.append(idx)
    return out


def face_array_len(p, k):
    """Volumes in one face array."""
    return 2 * k * p * p
