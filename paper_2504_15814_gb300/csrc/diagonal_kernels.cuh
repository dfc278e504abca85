// Diagonal (edge and vertex) ghost volumes of the fine patches.
//
// The paper's transfer carries no diagonal data (Sec. 2: only the face
// arrays of a hanging face are exchanged).  A fine patch whose stencils reach
// across its edges or corners also needs ghost volumes beyond the tangential
// extent of its subface.  They are filled here from the same coarse face
// array by the same rule as the ordinary ghost volumes: the ghost half of
// each subface's fine face array widened by k volumes on each tangential
// side, every volume reconstructed about its nearest coarse centre of the
// face array (on the face's edge when the volume lies past it, the offset
// then exceeding one fine spacing) with that centre's derivative stencils and
// Taylor's formula, or by the d-linear tensor product with linear
// extrapolation past the edge.  Inside the subface the values equal the
// ordinary interpolation.  Float64 arithmetic; one thread per (coarse
// centre, unknown) of each widened box.
#pragma once
#include "transfer_kernels.cuh"

namespace amr {

// Value at offset e (fine spacings, any integer) from x0 along one axis, by
// the line through x0 and the neighbour on e's side (xm below, xp above), or
// through x0 and the other neighbour where that side has none (extrapolation).
__device__ __forceinline__ double lerp_at(double xm, double x0, double xp, bool lo_edge, bool hi_edge, int e) {
  if (e == 0) return x0;
  const double f = (double)e * (1.0 / 3.0);  // offset in coarse spacings
  if (e < 0) return lo_edge ? x0 + f * (xp - x0) : x0 + f * (x0 - xm);
  return hi_edge ? x0 + f * (x0 - xm) : x0 + f * (xp - x0);
}

// d-linear value at offsets (en, e0, e1) from coarse centre (-1, a, b): the
// normal line on the 3 x 3 neighbour columns, then along t0, then along t1.
template <typename Src>
__device__ __forceinline__ double dlinear_at(const Src& S, int k, int p, int a, int b, int en, int e0, int e1) {
  const bool alo = a == 0, ahi = a == p - 1, blo = b == 0, bhi = b == p - 1;
  const int aidx[3] = {alo ? a : a - 1, a, ahi ? a : a + 1};
  const int bidx[3] = {blo ? b : b - 1, b, bhi ? b : b + 1};
  double A[3];
#pragma unroll
  for (int db = 0; db < 3; ++db) {
    double N[3];
#pragma unroll
    for (int da = 0; da < 3; ++da) {
      const double v1 = S(-1, aidx[da], bidx[db]);
      // normal offsets +1 (towards coarse layer 0), 0, -1 (towards layer -2, k >= 3)
      N[da] = en > 0 ? v1 + (1.0 / 3.0) * (S(0, aidx[da], bidx[db]) - v1)
                     : (en < 0 && k >= 3 ? v1 + (1.0 / 3.0) * (S(-2, aidx[da], bidx[db]) - v1) : v1);
    }
    A[db] = lerp_at(N[0], N[1], N[2], alo, ahi, e0);
  }
  return lerp_at(A[0], A[1], A[2], blo, bhi, e1);
}

// Evaluate the Taylor-m polynomial with coefficients C (fine units) at
// integer offsets (en, e0, e1).
template <int M>
__device__ __forceinline__ double taylor_at(const double (&C)[M + 1][M + 1][M + 1], int en, int e0, int e1) {
  double v = 0.0, xn = 1.0;
#pragma unroll
  for (int x = 0; x <= M; ++x) {
    double x1p = 1.0;
#pragma unroll
    for (int y = 0; x + y <= M; ++y) {
      double x2p = 1.0;
#pragma unroll
      for (int z = 0; x + y + z <= M; ++z) {
        v = fma(C[x][y][z], xn * x1p * x2p, v);
        x2p *= (double)e1;
      }
      x1p *= (double)e0;
    }
    xn *= (double)en;
  }
  return v;
}

// Fine global indices [lo, hi] along one tangential axis whose nearest coarse
// centre is a, within the widened box [box_lo, box_hi] (past the face's edges
// the edge centres take every remaining index).
__device__ __forceinline__ void centre_span(int a, int p, int box_lo, int box_hi, int& lo, int& hi) {
  lo = a == 0 ? box_lo : max(3 * a, box_lo);
  hi = a == p - 1 ? box_hi : min(3 * a + 2, box_hi);
}

// One tile = one fine face array (slot) of one item and a chunk of unknowns.
// One thread per (coarse centre, unknown): the centre's Taylor coefficients
// (or its d-linear neighbourhood) once, then every widened-box volume whose
// nearest centre it is.  diag layout, from diag_off[item]:
// ((((slot k + g) W + q1 + k) W + q0 + k) U + u with W = p + 2k, ghost layer g
// (0 next to the interface), tangential local indices q0, q1 in [-k, p + k).
__global__ void __launch_bounds__(256) interp_diagonal_kernel(const amr_transfer_item* __restrict__ items,
                                                              const AdjointTile* __restrict__ tiles, int U,
                                                              const int64_t* __restrict__ diag_off,
                                                              const double* __restrict__ coarse,
                                                              double* __restrict__ diag) {
  const AdjointTile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.index];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  const int sub = it.subface < 0 ? t.slot : it.subface;
  const int s0 = sub % 3, s1 = sub / 3;
  const int W = p + 2 * k, nu = t.nu;
  double* out = diag + diag_off[t.index] + (int64_t)t.slot * k * W * W * U;
  const double* cb = coarse + it.coarse_offset;
  // widened box in fine global indices, and the centres it reaches
  const int lo0 = s0 * p - k, hi0 = s0 * p + p + k - 1, lo1 = s1 * p - k, hi1 = s1 * p + p + k - 1;
  const int a_lo = lo0 < 0 ? 0 : min(lo0 / 3, p - 1), a_hi = min(hi0 / 3, p - 1);
  const int b_lo = lo1 < 0 ? 0 : min(lo1 / 3, p - 1), b_hi = min(hi1 / 3, p - 1);
  const int na = a_hi - a_lo + 1, nb = b_hi - b_lo + 1;
  for (int e = threadIdx.x; e < na * nb * nu; e += blockDim.x) {
    const int u = t.u0 + e % nu, c = e / nu;
    const int a = a_lo + c % na, b = b_lo + c / na;
    int g0a, g0b, g1a, g1b;
    centre_span(a, p, lo0, hi0, g0a, g0b);
    centre_span(b, p, lo1, hi1, g1a, g1b);
    auto S = [&](int j, int aa, int bb) -> double { return __ldg(cb + frame_vol(fr, j, aa, bb) * U + u); };
    auto put = [&](int g, int g0, int g1, double v) {
      out[((int64_t)(g * W + g1 - s1 * p + k) * W + (g0 - s0 * p + k)) * U + u] = v;
    };
    if (m == 1) {
      for (int g = 0; g < k; ++g)
        for (int g1 = g1a; g1 <= g1b; ++g1)
          for (int g0 = g0a; g0 <= g0b; ++g0)
            put(g, g0, g1, dlinear_at(S, k, p, a, b, 1 - g, g0 - (3 * a + 1), g1 - (3 * b + 1)));
    } else if (m == 3) {
      double C[4][4][4];
      taylor_interp_coeffs<3, double>(S, c_wt_interp, k, p, a, b, S(-1, a, b), -1, C);
      for (int g = 0; g < k; ++g)
        for (int g1 = g1a; g1 <= g1b; ++g1)
          for (int g0 = g0a; g0 <= g0b; ++g0) put(g, g0, g1, taylor_at<3>(C, 1 - g, g0 - (3 * a + 1), g1 - (3 * b + 1)));
    } else {
      double C[3][3][3];
      taylor_interp_coeffs<2, double>(S, c_wt_interp, k, p, a, b, S(-1, a, b), -1, C);
      for (int g = 0; g < k; ++g)
        for (int g1 = g1a; g1 <= g1b; ++g1)
          for (int g0 = g0a; g0 <= g0b; ++g0) put(g, g0, g1, taylor_at<2>(C, 1 - g, g0 - (3 * a + 1), g1 - (3 * b + 1)));
    }
  }
}

}  // namespace amr
