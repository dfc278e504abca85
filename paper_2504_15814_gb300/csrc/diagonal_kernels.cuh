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
// ordinary interpolation.  Float64 arithmetic; one thread per (volume,
// unknown), derivatives recomputed per volume (the widened boxes are small
// next to the face arrays).
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

// One tile = one fine face array (slot) of one item and a chunk of unknowns.
// diag layout, from diag_off[item]: ((((slot k + g) W + q1 + k) W + q0 + k) U + u
// with W = p + 2k, ghost layer g (0 next to the interface), tangential local
// indices q0, q1 in [-k, p + k).
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
  const int W = p + 2 * k, npos = k * W * W, nu = t.nu;
  double* out = diag + diag_off[t.index] + (int64_t)t.slot * npos * U;
  const double* cb = coarse + it.coarse_offset;
  for (int e = threadIdx.x; e < npos * nu; e += blockDim.x) {
    const int u = t.u0 + e % nu, pos = e / nu;
    const int q0 = pos % W - k, q1 = (pos / W) % W - k, g = pos / (W * W);
    // fine global tangential indices; nearest coarse centre (clamped to the
    // face) and the offsets from it, in fine spacings
    const int g0 = s0 * p + q0, g1 = s1 * p + q1;
    const int a = g0 < 0 ? 0 : min(g0 / 3, p - 1);
    const int b = g1 < 0 ? 0 : min(g1 / 3, p - 1);
    const int e0 = g0 - (3 * a + 1), e1 = g1 - (3 * b + 1), en = 1 - g;
    auto S = [&](int j, int aa, int bb) -> double { return __ldg(cb + frame_vol(fr, j, aa, bb) * U + u); };
    double v;
    if (m == 1) {
      v = dlinear_at(S, k, p, a, b, en, e0, e1);
    } else {
      double C[4][4][4];
      double xn = 1.0;
      if (m == 3) {
        double C3[4][4][4];
        taylor_interp_coeffs<3, double>(S, c_wt_interp, k, p, a, b, S(-1, a, b), -1, C3);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) C[x][y][z] = C3[x][y][z];
      } else {
        double C2[3][3][3];
        taylor_interp_coeffs<2, double>(S, c_wt_interp, k, p, a, b, S(-1, a, b), -1, C2);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) C[x][y][z] = (x < 3 && y < 3 && z < 3) ? C2[x][y][z] : 0.0;
      }
      // sum over |alpha| <= m of C_alpha en^x e0^y e1^z
      v = 0.0;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        double x1p = 1.0;
#pragma unroll
        for (int y = 0; x + y < 4; ++y) {
          double x2p = 1.0;
#pragma unroll
          for (int z = 0; x + y + z < 4; ++z) {
            v = fma(C[x][y][z], xn * x1p * x2p, v);
            x2p *= (double)e1;
          }
          x1p *= (double)e0;
        }
        xn *= (double)en;
      }
    }
    out[(int64_t)pos * U + u] = v;
  }
}

}  // namespace amr
