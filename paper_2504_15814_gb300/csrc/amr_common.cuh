// Geometry, window rule and work-tile types shared by the host operator
// builder and the sm_103a kernels.
//
// Reference frame of a face (the paper, Sec. 4.1, maps all six face
// configurations onto one reference face by rotation and mirroring; here that
// mapping is index arithmetic, with no copy):
//   * signed normal layer j in [-k, k-1]: j < 0 on the coarse patch's own
//     side, j = -1 and j = 0 touch the interface.  Face-array normal index
//     i_n = j + k for faces 0..2 (coarse on the low side) and k - 1 - j for
//     faces 3..5 (coarse on the high side, mirrored);
//   * tangential indices a (along t0) and b (along t1) are never mirrored;
//   * coarse centre of layer j at (j + 1/2) H, fine layer i at (i + 1/2) h,
//     h = H / 3; coarse tangential a at (a + 1/2) H, fine global tangential
//     g = s_t p + q at (g + 1/2) h, so fine g coincides with coarse g / 3
//     exactly when g = 3a + 1;
//   * coarse a covers fine 3a .. 3a+2.  When p is not a multiple of 3 a
//     subface boundary can cut a coarse volume: its children then lie in two
//     fine face arrays, and it is restricted by the subface holding 3a + 1.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/amr_transfer.h"

namespace amr {

// One unit of device work: a rectangle of coarse columns of one subface of
// one item, and a contiguous range of unknowns.
//   interpolation: the coarse centres (a, b) of every centre layer (-1, and
//                  -2 for overlaps 4, 5) whose fine children lie in the subface;
//   restriction:   the coarse halo columns (a, b) over the subface.
struct Tile {
  int32_t item;
  int8_t sub;     // subface 0..8
  int8_t slot;    // index of the subface's fine face array within the item (0 or sub)
  int8_t na, nb;  // columns along t0, t1
  int16_t a0, b0; // first coarse tangential index
  int16_t u0, nu; // unknown range
};
static_assert(sizeof(Tile) == 16, "Tile must stay 16 bytes");

struct FaceFrame {
  int64_t s_n;     // signed volume stride of one normal layer step (j -> j+1)
  int64_t base_n;  // volume offset of layer j = 0
  int64_t s_t0, s_t1;
  int64_t vols;    // volumes per face array
};

__host__ __device__ inline FaceFrame face_frame(int face, int p, int k) {
  // extents: 2k along the normal axis n = face % 3, p along the others;
  // strides of a lexicographic box with x fastest (selects, no local arrays)
  const int n = face % 3;
  const int64_t ex = n == 0 ? 2 * k : p, ey = n == 1 ? 2 * k : p, ez = n == 2 ? 2 * k : p;
  const int64_t sy = ex, sz = ex * ey;
  const int64_t sn = n == 0 ? 1 : (n == 1 ? sy : sz);
  FaceFrame f;
  f.s_n = (face < 3) ? sn : -sn;
  f.base_n = (face < 3) ? (int64_t)k * sn : (int64_t)(k - 1) * sn;
  f.s_t0 = n == 0 ? sy : 1;   // t0 = y for normal x, else x
  f.s_t1 = n == 2 ? sy : sz;  // t1 = y for normal z, else z
  f.vols = ex * ey * ez;
  return f;
}

__host__ __device__ inline int64_t frame_vol(const FaceFrame& f, int j, int a, int b) {
  return f.base_n + (int64_t)j * f.s_n + (int64_t)a * f.s_t0 + (int64_t)b * f.s_t1;
}

// Window rule of the derivative stencils (the paper's appendix "Stencil
// Structure": centred where possible, biased towards the centre of the
// pre-image patch at its edges, no diagonal data).  A derivative that must be
// exact up to degree E along this axis uses the smallest odd number of
// consecutive centres L >= E+1, centred on c and shifted inward to fit
// [lo, hi]; a range shorter than that but holding E+1 centres is used whole.
// The host rejects ranges shorter than E+1.
__host__ __device__ inline void stencil_window(int c, int lo, int hi, int E, int& start, int& len) {
  const int need = E + 1;
  const int odd = need | 1;
  const int avail = hi - lo + 1;
  if (avail < odd) {
    start = lo;
    len = avail;
  } else {
    int s = c - odd / 2;
    if (s < lo) s = lo;
    if (s > hi - odd + 1) s = hi - odd + 1;
    start = s;
    len = odd;
  }
}

// Length of the window used for pure derivatives (exact to degree m) and for
// mixed derivatives (exact to degree <= 2 along each axis: 3 points).
__host__ __device__ inline int pure_exactness(int order) { return order; }
__host__ __device__ inline int mixed_exactness(int order) { return order == 3 ? 2 : 1; }

// Coarse tangential indices [lo, hi) restricted by subface position s: those
// whose coincident fine index 3a + 1 lies in [s p, s p + p).
__host__ __device__ inline void owned_range(int s, int p, int& lo, int& hi) {
  lo = (s * p + 1) / 3;
  hi = (s * p + p + 1) / 3;
}

// Coarse tangential indices [lo, hi) with at least one fine child in subface
// position s (interpolation sources of that subface).
__host__ __device__ inline void covering_range(int s, int p, int& lo, int& hi) {
  lo = (s * p) / 3;
  hi = (s * p + p - 1) / 3 + 1;
}

struct IRange { int lo, hi; };

// Inclusive index range, along one axis holding [lo, hi], of every centre the
// derivative stencils of the coarse centres [c0, c1] touch (Taylor-m; windows
// move monotonically with the centre, so the end centres bound the union).
__host__ __device__ inline IRange taylor_union(int c0, int c1, int lo, int hi, int order) {
  int s, l, lo_u = c0, hi_u = c1;
  const int E[2] = {pure_exactness(order), mixed_exactness(order)};
  for (int q = 0; q < 2; ++q) {
    const int c = q == 0 ? c0 : c1;
    for (int e = 0; e < 2; ++e) {
      stencil_window(c, lo, hi, E[e], s, l);
      lo_u = s < lo_u ? s : lo_u;
      hi_u = s + l - 1 > hi_u ? s + l - 1 : hi_u;
    }
  }
  IRange r{lo_u, hi_u};
  return r;
}

// Deepest overlap served.  Fine ghost layer -1 - g (g = 0..k-1) lies inside
// coarse layer -1 - g / 3, so overlaps 4 and 5 put the fine ghost layers
// -4..-k under a second layer of interpolation centres (coarse layer -2).
constexpr int kMaxOverlap = 5;
// Coarse layers holding interpolation centres (layers -1, ..., -centre_layers).
__host__ __device__ inline int centre_layers(int k) { return (k + 2) / 3; }
// Fine ghost layers below centre layer m (coarse layer -1 - m): fine layers
// -1 - 3m - ii for ii < child_layers(k, m).
__host__ __device__ inline int child_layers(int k, int m) { return k - 3 * m < 3 ? k - 3 * m : 3; }

// Region of the coarse face array one interpolation tile reads: signed normal
// layers rn, tangential ranges ra (t0) and rb (t1).  Each centre layer cl
// reads layers cl and cl + 1 for d-linear (and cl - 1 when its three child
// layers reach below it); Taylor reads the union of the derivative windows of
// all centre layers.
__host__ __device__ inline void interp_region(int p, int k, int order, int a0, int na, int b0, int nb,
                                              IRange& rn, IRange& ra, IRange& rb) {
  const int cl_lo = -centre_layers(k);
  if (order == AMR_ORDER_DLINEAR) {
    rn.lo = child_layers(k, centre_layers(k) - 1) >= 3 ? cl_lo - 1 : cl_lo; rn.hi = 0;
    ra.lo = a0 > 0 ? a0 - 1 : 0; ra.hi = a0 + na < p ? a0 + na : p - 1;
    rb.lo = b0 > 0 ? b0 - 1 : 0; rb.hi = b0 + nb < p ? b0 + nb : p - 1;
  } else {
    rn = taylor_union(cl_lo, -1, -k, k - 1, order);
    ra = taylor_union(a0, a0 + na - 1, 0, p - 1, order);
    rb = taylor_union(b0, b0 + nb - 1, 0, p - 1, order);
  }
}

// Weight table layout: 1-D derivative weights for windows of L = 3, 4, 5
// consecutive unit-spaced centres, expansion point at position pos in the
// window, derivative order r = 1..3, stored as lambda / r! (the Taylor
// coefficient form).  Entry (L, pos, r, i) at wt_offset(L) + (pos*3 + r-1)*L + i.
__host__ __device__ inline int wt_offset(int L) { return L == 3 ? 0 : (L == 4 ? 27 : 75); }
constexpr int WT_SIZE = 150;

// Denominator that makes every entry (L, pos, r, .) of the Taylor-coefficient
// weight table an integer: 2 for the 3-point windows (Taylor-2 lines and all
// mixed windows), 12, 24, 12 for r = 1, 2, 3 on the 4- and 5-point windows
// of the Taylor-3 lines.
__host__ __device__ inline int fixed_den(int L, int r) { return L == 3 ? 2 : (r == 2 ? 24 : 12); }

// Least-squares line weights of the d-linear restriction, per overlap k,
// coarse halo layer j < k and fine layer slot i < kMaxOverlap (the fine
// patch's own layers 0..k-1, or layers -1, 0 when k = 1).
constexpr int LS_SIZE = kMaxOverlap * kMaxOverlap * kMaxOverlap;
__host__ __device__ inline int ls_index(int k, int j, int i) {
  return ((k - 1) * kMaxOverlap + j) * kMaxOverlap + i;
}

// Combined Taylor restriction weights: coarse halo layer j >= 1 of a face with
// overlap k (2..kMaxOverlap) and order m (2 or 3) is sum_i W[i] u(fine layer
// s + i) over the derivative window (s, L) about fine layer k - 1 (Sec. 3:
// Taylor about the nearest fine cell, extrapolated by (3j + 2 - k) h), for
// the finite-difference (scheme 0) or least-squares (scheme 1) derivatives.
constexpr int RW_SIZE = 2 * 2 * (kMaxOverlap - 1) * (kMaxOverlap - 1) * 5;
__host__ __device__ inline int rw_index(int order, int k, int j, int scheme = 0) {
  return ((((scheme * 2 + order - 2) * (kMaxOverlap - 1) + (k - 2)) * (kMaxOverlap - 1)) + (j - 1)) * 5;
}

// Least-squares interpolation (scheme 1) in the factorised kernel: the
// derivatives of a coarse centre are W^T d over the values d of the
// finite-difference stencils' slots -- the three pure lines (slot 5 d + i,
// point ps[d] + i along axis d, i < the window length) and the 3x3x3 box of
// the mixed windows (slot 15 + (q * 3 + j) * 3 + i, point (ms0 + i, ms1 + j,
// ms2 + q)).  W depends on where the centre sits along each tangential axis
// (ls_class: first, second, interior, second-last, last), so a table block
// per (p, k, order) holds LS_CLASSES slot x derivative matrices, then the
// per-class column sums of W.
constexpr int LS_SLOTS = 42;
constexpr int LS_NALPHA = 19;  // derivatives 0 < |alpha| <= 3
constexpr int LS_CLASSES = 25;
constexpr int LS_BLOCK = LS_CLASSES * (LS_SLOTS + 1) * LS_NALPHA;
__host__ __device__ inline int ls_class(int a, int p) { return a < 2 ? a : (a > p - 3 ? 4 - (p - 1 - a) : 2); }
__host__ __device__ inline int ls_class_rep(int cls, int p) { return cls < 3 ? cls : p - 5 + cls; }

}  // namespace amr
