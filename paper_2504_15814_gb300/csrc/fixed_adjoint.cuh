// Factorised adjoints of the finite-difference operators.
//
// P^T (interpolation adjoint), exact fixed point.  The forward operator
// evaluates, per coarse centre c, the Taylor coefficients C_alpha = sum_j
// w_alpha,j x_j (Sec. 3; the full stencil weights, the centre's included,
// since every derivative stencil's weights sum to zero) and the children
// v_e = x_c + sum_alpha e^alpha C_alpha.  Its transpose, per centre:
//   gamma_0 = sum_e g_e,  gamma_alpha = sum_e e^alpha g_e   (moments of the
//   27 child gradients, separable: along each axis the values at -1, 0, +1
//   give the sum, the difference and the outer sum),
//   then x_c += gamma_0 and x_j += w_alpha,j gamma_alpha over the stencils
//   (the transposed pure lines and the transposed 3x3x3 box collapse).
// Contributions of neighbouring centres overlap, so they are summed in a
// shared-memory accumulator; the gradients are first rounded onto a common
// grid 2^-s per coarse array and unknown (|n| < 2^44 over every ghost
// gradient of the group), after which everything is exact int64 arithmetic
// with the integer stencil numerators scaled to the common denominator 648
// -- the sum is exact and independent of the order of the integer atomic
// adds, so the result is deterministic.  Each coarse value is T q / 648,
// rounded once (T / 81 to an integer, then an exact power-of-two scale).
// Error: the rounding of the inputs, below (row sum of |P^T|) 2^-45 of the
// largest ghost gradient.
//
// R^T (restriction adjoint), float64.  Each coarse halo column restricts
// from its coincident fine column only (injection at coarse layer 0,
// combined extrapolation weights W_j for the deeper layers), so R^T of one
// column is a 5 x 3 product: fine layer s + i of the window receives
// [s + i == 1] g_0 + sum_{j >= 1} W_j[i] g_j.  R^T overwrites the whole fine
// buffer, so the kernel writes every value of its fine face arrays: zeros
// by flat 16-byte stores, then the window values.
#pragma once
#include "fixed_kernels.cuh"

namespace amr {

constexpr int kAdjBits = 44;  // quantized gradients satisfy |n| < 2^44
constexpr int kAdjThreads = 256;

// L2 eviction policy for loads that are the last use of their lines (PTX
// createpolicy), so that they do not displace lines other CTAs read again.
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double ld_hint(const double* ptr, unsigned long long pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
  return v;
}

// round(x 2^s) for a float64 x with |x| < 2^(44 - s): exact shift of the
// significand (no float64 instruction), ties away from zero.  The bound puts
// x 2^s = m 2^-r with r = 1075 - s - E >= 9, so the shift is always to the
// right: floor(m / 2^(r-1)), plus one, halved.  Subnormal x give 0.
__device__ __forceinline__ long long quantize_pow2(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ffull);
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  const int r1 = min(1074 - s - E, 63);  // r - 1 >= 8; m < 2^53 gives 0 from 53 on
  const unsigned long long t = E ? (m >> r1) : 0ull;
  const long long n = (long long)((t + 1ull) >> 1);
  return (long long)(b >> 63) ? -n : n;
}

// T * 2^-s / 648 as float64: T / 81 rounded to the nearest integer (ties
// away from zero), then scaled by 2^-(s + 3) exactly.
__device__ __forceinline__ double adj_to_f64(long long T, int s, uint32_t ovf_hi) {
  const unsigned long long sg = (unsigned long long)(T >> 63);
  const unsigned long long mag = ((unsigned long long)T ^ sg) - sg;
  // floor((mag + 40) / 81) by a multiply-high with the reciprocal 2^70 / 81
  // (exact for mag + 40 < 2^63: the reciprocal's error stays below 1/81)
  const unsigned long long num = mag + 40ull;
  unsigned long long q = __umul64hi(num, 0xCA4587E6B74F0329ull) >> 6;  // ceil(2^70 / 81)
  if (q * 81ull > num) --q;
  const long long Q = (long long)((q ^ sg) - sg);
  return fixed_to_f64(Q, s + 3, ovf_hi);
}

// Moments of one axis: values at -1, 0, +1 -> (sum, difference, outer sum):
// the transposed even/odd evaluation (order 0, odd orders, even orders >= 2).
struct Mom3 { long long s0, od, ev; };
__device__ __forceinline__ Mom3 mom3(long long m, long long z, long long p) {
  Mom3 r;
  r.ev = m + p;
  r.s0 = r.ev + z;
  r.od = p - m;
  return r;
}
__device__ __forceinline__ long long mom_pick(const Mom3& v, int r) { return r == 0 ? v.s0 : ((r & 1) ? v.od : v.ev); }

// 3-point first-derivative numerator weights (denominator 2) at position pos,
// for point i: centred (-1, 0, 1), pos 0 (-3, 4, -1), pos 2 (1, -4, 3).
__device__ __forceinline__ int w13(int pos, int i) {
  return i == 0 ? (pos == 0 ? -3 : (pos == 1 ? -1 : 1)) : (i == 1 ? (pos == 0 ? 4 : (pos == 1 ? 0 : -4))
                                                                  : (pos == 0 ? -1 : (pos == 1 ? 1 : 3)));
}
__device__ __forceinline__ int w23(int i) { return i == 1 ? -2 : 1; }

// ---------------------------------------------------------------------------
// Transpose of one centre's Taylor-m (m = 2, 3) interpolation: scatters
// 648 x (the gradient contributions) of one unknown into the accumulator.
// gmom(x, y, z) returns the moment of the child gradients for the monomial
// e_n^x e0^y e1^z (x, y, z: derivative orders); add(j, a', b', v) adds v to
// the accumulator at coarse (signed normal layer j, a', b').
// ---------------------------------------------------------------------------
template <int M, typename Mom, typename Add>
__device__ __forceinline__ void taylor_fixed_adjoint(const Mom& gmom, const Add& add, int k, int p, int a, int b) {
  const int c[3] = {-1, a, b};
  const int lo[3] = {-k, 0, 0};
  const int hi[3] = {k - 1, p - 1, p - 1};
  int ps[3], pl[3], ms[3], ml[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    stencil_window(c[d], lo[d], hi[d], pure_exactness(M), ps[d], pl[d]);
    stencil_window(c[d], lo[d], hi[d], mixed_exactness(M), ms[d], ml[d]);
  }
  constexpr int GS = M == 3 ? 1 : 18;  // 648 / G
  add(-1, a, b, 648 * gmom(0, 0, 0));
  // pure lines: point i of the window gets sum_r M_r N_r[i] gamma_r
  // (Taylor-3: M_r = 18, 3, 2 over numerators 12, 24, 12; Taylor-2: 6, 2 over 2)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int pos = c[d] - ps[d], L = pl[d];
    long long g[3];
#pragma unroll
    for (int r = 1; r <= M; ++r) g[r - 1] = gmom(d == 0 ? r : 0, d == 1 ? r : 0, d == 2 ? r : 0);
    const long long m1 = (M == 3 ? 18 : 6) * GS * g[0], m2 = (M == 3 ? 3 : 2) * GS * g[1];
    const long long m3 = M == 3 ? 2 * g[2] : 0;
    const int32_t* w = c_fxw + wt_offset(L) + pos * 3 * L;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (i < L) {
        long long v = (long long)w[i] * m1 + (long long)w[L + i] * m2;
        if (M == 3) v += (long long)w[2 * L + i] * m3;
        int x[3] = {c[0], c[1], c[2]};
        x[d] = ps[d] + i;
        add(x[0], x[1], x[2], v);
      }
    }
  }
  // mixed derivatives: transpose of the box collapse (normal, then t0, then
  // t1) with scalings 648 / (4 9) = 18 for (1,1), 648 / (4 27) = 6 for (2,1),
  // 648 / (8 27) = 3 for (1,1,1) (Taylor-3) and 36 / 36 = 1 for (1,1) (Taylor-2)
  const int sa = c[1] - ms[1], sb = c[2] - ms[2];
  const long long g110 = (M == 3 ? 18 : GS) * gmom(1, 1, 0), g101 = (M == 3 ? 18 : GS) * gmom(1, 0, 1);
  const long long g011 = (M == 3 ? 18 : GS) * gmom(0, 1, 1);
  long long g210 = 0, g120 = 0, g201 = 0, g102 = 0, g021 = 0, g012 = 0, g111 = 0;
  if (M == 3) {
    g210 = 6 * gmom(2, 1, 0); g120 = 6 * gmom(1, 2, 0); g201 = 6 * gmom(2, 0, 1);
    g102 = 6 * gmom(1, 0, 2); g021 = 6 * gmom(0, 2, 1); g012 = 6 * gmom(0, 1, 2);
    g111 = 3 * gmom(1, 1, 1);
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int b1 = w13(sb, q), b2 = w23(q);
    const bool qs = q == sb;
    const long long dP11 = (qs ? g110 : 0) + (M == 3 ? b1 * g111 : 0);
    const long long dP10 = b1 * g101 + (M == 3 ? b2 * g102 : 0);
    const long long dP01 = b1 * g011 + (M == 3 ? b2 * g012 : 0);
    const long long dP21 = qs ? g210 : 0, dP12 = qs ? g120 : 0;
    const long long dP20 = b1 * g201, dP02 = b1 * g021;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int a1 = w13(sa, j), a2 = w23(j);
      const bool js = j == sa;
      const long long ds1 = a1 * dP11 + (js ? dP10 : 0) + (M == 3 ? a2 * dP12 : 0);
      const long long ds2 = M == 3 ? (js ? dP20 : 0) + a1 * dP21 : 0;
      const long long dx1 = a1 * dP01 + (M == 3 ? a2 * dP02 : 0);
      // normal window centred on layer -1: s1 = x2 - x0, s2 = x0 - 2 x1 + x2
      add(ms[0], ms[1] + j, ms[2] + q, ds2 - ds1);
      add(ms[0] + 1, ms[1] + j, ms[2] + q, dx1 - 2 * ds2);
      add(ms[0] + 2, ms[1] + j, ms[2] + q, ds1 + ds2);
    }
  }
}

// Transpose of one centre's d-linear interpolation (G = 27, scaled by 24 to
// the common 648): the transposed 1-D lerps along t1, t0 and the normal.
template <typename Grad, typename Add>
__device__ __forceinline__ void dlinear_fixed_adjoint(const Grad& grad, const Add& add, int k, int p, int a, int b) {
  const bool alo = a == 0, ahi = a == p - 1, blo = b == 0, bhi = b == p - 1;
  const int aidx[3] = {alo ? a : a - 1, a, ahi ? a : a + 1};
  const int bidx[3] = {blo ? b : b - 1, b, bhi ? b : b + 1};
  // transpose of lerp3: (gm, gz, gp) -> gradients of (xm, x0, xp)
  auto tl = [](long long gm, long long gz, long long gp, bool le, bool he, long long& dm, long long& d0, long long& dp) {
    d0 = 3 * gz + (le ? 4 : 2) * gm + (he ? 4 : 2) * gp;
    dm = (le ? 0 : gm) - (he ? gp : 0);
    dp = (he ? 0 : gp) - (le ? gm : 0);
  };
  long long dN[3][3][3];  // [ii][da][db]
#pragma unroll
  for (int ii = 0; ii < 3; ++ii)
#pragma unroll
    for (int da = 0; da < 3; ++da)
#pragma unroll
      for (int db = 0; db < 3; ++db) dN[ii][da][db] = 0;
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) {
    if (ii >= k) break;
    long long dA[3][3];  // [e0][db]
#pragma unroll
    for (int e0 = 0; e0 < 3; ++e0)
      tl(grad(ii, e0 - 1, -1), grad(ii, e0 - 1, 0), grad(ii, e0 - 1, 1), blo, bhi, dA[e0][0], dA[e0][1], dA[e0][2]);
#pragma unroll
    for (int db = 0; db < 3; ++db) tl(dA[0][db], dA[1][db], dA[2][db], alo, ahi, dN[ii][0][db], dN[ii][1][db], dN[ii][2][db]);
  }
#pragma unroll
  for (int da = 0; da < 3; ++da)
#pragma unroll
    for (int db = 0; db < 3; ++db) {
      // N0 = 2 v(-1) + v(0), N1 = 3 v(-1), N2 = 2 v(-1) + v(-2) (k >= 3)
      const long long d1 = 2 * dN[0][da][db] + 3 * dN[1][da][db] + (k >= 3 ? 2 * dN[2][da][db] : 0);
      add(-1, aidx[da], bidx[db], 24 * d1);
      add(0, aidx[da], bidx[db], 24 * dN[0][da][db]);
      if (k >= 3) add(-2, aidx[da], bidx[db], 24 * dN[2][da][db]);
    }
}

// ---------------------------------------------------------------------------
// First step of the fixed-point P^T: per group of items sharing a coarse face
// array and chunk of <= 32 unknowns, the largest biased exponent of the
// group's ghost gradients per unknown (the grid of the exact accumulation).
// It is left, as an integer, in the first volume of the group's coarse face
// array (g_coarse, which interp_adjoint_fixed_kernel reads and then
// overwrites).  A separate light kernel streams the gradients at high
// occupancy; inside the accumulation kernel (two CTAs per SM) the same scan
// ran at about half the bandwidth.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads)
    adjoint_emax_kernel(const amr_transfer_item* __restrict__ items, const AdjointTile* __restrict__ tiles,
                        const int32_t* __restrict__ group_ptr, const int32_t* __restrict__ group_items, int U,
                        const double* __restrict__ g_fine, double* __restrict__ g_coarse) {
  __shared__ int s_emax[32];
  const AdjointTile t = tiles[blockIdx.x];
  const int m0 = group_ptr[t.index], m1 = group_ptr[t.index + 1];
  const amr_transfer_item first = items[group_items[m0]];
  const int p = first.patch_size, k = first.overlap;
  const FaceFrame fr = face_frame(first.face, p, k);
  const int64_t arr = fr.vols * U;
  const int nu = t.nu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nu > 32) return;
  if (threadIdx.x < 32) s_emax[threadIdx.x] = 0;
  __syncthreads();
  const int gs_a = (int)fr.s_t0 * U;
  // a warp takes one ghost row (p volumes along t0) at a time
  if (lane < nu) {
    int emax = 0;
    for (int mi = m0; mi < m1; ++mi) {
      const amr_transfer_item it = items[group_items[mi]];
      const int nsub = it.subface < 0 ? 9 : 1;
      const int nrow = nsub * k * p;  // rows (slot, ghost layer g, q1)
      int slot = 0, g = 0, q1 = warp;  // row index warp, stepping by nw
      while (q1 >= p) { q1 -= p; if (++g == k) { g = 0; ++slot; } }
      // two rows per iteration, their loads in flight together
      for (int row = warp; row < nrow; row += 2 * nw) {
        const double* src0 = g_fine + it.fine_offset + slot * arr + frame_vol(fr, -1 - g, 0, q1) * U + t.u0 + lane;
        q1 += nw;
        while (q1 >= p) { q1 -= p; if (++g == k) { g = 0; ++slot; } }
        const bool two = row + nw < nrow;
        const double* src1 = two ? g_fine + it.fine_offset + slot * arr + frame_vol(fr, -1 - g, 0, q1) * U + t.u0 + lane
                                 : src0;
        q1 += nw;
        while (q1 >= p) { q1 -= p; if (++g == k) { g = 0; ++slot; } }
        constexpr int CH = 12;
        for (int q0 = 0; q0 < p; q0 += CH) {
          double x[2][CH];
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            x[0][c] = q0 + c < p ? __ldg(src0 + (q0 + c) * gs_a) : 0.0;
            x[1][c] = q0 + c < p ? __ldg(src1 + (q0 + c) * gs_a) : 0.0;
          }
#pragma unroll
          for (int c = 0; c < CH; ++c)
            emax = max(emax, (int)(max(__double_as_longlong(x[0][c]) >> 52 & 0x7ff, __double_as_longlong(x[1][c]) >> 52 & 0x7ff)));
        }
      }
    }
    atomicMax(&s_emax[lane], emax);
  }
  __syncthreads();
  if (threadIdx.x < nu)
    reinterpret_cast<long long*>(g_coarse)[first.coarse_offset + t.u0 + threadIdx.x] = s_emax[threadIdx.x];
}

// ---------------------------------------------------------------------------
// g_coarse = P^T g_fine, fixed point, for one group of items sharing a
// coarse face array (finite-difference items, p a multiple of 3) and a chunk
// of <= 32 unknowns, after adjoint_emax_kernel has left the grid exponents
// in the array.  One warp per coarse centre, lane = unknown: the centre's
// child gradients rounded onto the grid, reduced to moments and scattered
// through the transposed stencils into the shared-memory accumulator (rows
// rlo..rhi: the union of the items' normal stencil ranges); then every value
// of the group's coarse face array is written (zero where nothing reaches).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads, 2)
    interp_adjoint_fixed_kernel(const amr_transfer_item* __restrict__ items, const AdjointTile* __restrict__ tiles,
                                const int32_t* __restrict__ group_ptr, const int32_t* __restrict__ group_items, int U,
                                const double* __restrict__ g_fine, double* __restrict__ g_coarse) {
  extern __shared__ double smem_raw[];
  long long* acc = reinterpret_cast<long long*>(smem_raw);
  const AdjointTile t = tiles[blockIdx.x];
  const int m0 = group_ptr[t.index], m1 = group_ptr[t.index + 1];
  const amr_transfer_item first = items[group_items[m0]];
  const int p = first.patch_size, k = first.overlap;
  const FaceFrame fr = face_frame(first.face, p, k);
  const int64_t arr = fr.vols * U;
  int rlo = 0, rhi = -1;  // union of the items' normal stencil ranges
  for (int mi = m0; mi < m1; ++mi) {
    IRange rn, ra, rb;
    interp_region(p, k, items[group_items[mi]].order, 0, p, 0, p, rn, ra, rb);
    rlo = min(rlo, rn.lo);
    rhi = max(rhi, rn.hi);
  }
  const int NJ = rhi - rlo + 1, npts = NJ * p * p;
  const int nu = t.nu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t dyn_smem;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
  if ((uint32_t)npts * 32u * 8u > dyn_smem || nu > 32) return;  // the host sizes the launch; never stage out of bounds
  for (int i = threadIdx.x; i < npts * 32; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  const int gs_n = (int)fr.s_n * U, gs_a = (int)fr.s_t0 * U, gs_b = (int)fr.s_t1 * U;
  // the largest biased exponent of the group's ghost gradients for this
  // lane's unknown, left by adjoint_emax_kernel in the first volume of the
  // group's coarse face array (read before this CTA writes it)
  const int E = lane < nu ? (int)reinterpret_cast<const long long*>(g_coarse)[first.coarse_offset + t.u0 + lane] : 0;
  const bool finite = E < 2047;
  const int s = kAdjBits - (max(E, 62) - 1022);  // |g| < 2^(E - 1022) -> |n| < 2^44
  // per item and coarse centre (one warp), the transposed operator
  if (lane < nu) {
    for (int mi = m0; mi < m1; ++mi) {
      const amr_transfer_item it = items[group_items[mi]];
      const int m = it.order;
      int alo = 0, ahi = p, blo = 0, bhi = p;
      if (it.subface >= 0) {
        covering_range(it.subface % 3, p, alo, ahi);
        covering_range(it.subface / 3, p, blo, bhi);
      }
      const int na = ahi - alo, ntask = na * (bhi - blo);
      int a = alo + warp, b = blo;
      while (a >= ahi) { a -= na; ++b; }
      for (int e = warp; e < ntask; e += nw, a += nw) {
        while (a >= ahi) { a -= na; ++b; }
        // subface of the centre's children: 3a / p along each axis (p a multiple of 3)
        const float inv_p = 1.0f / (float)p;
        const int s0 = it.subface >= 0 ? it.subface % 3 : (int)(((float)a + 0.5f) * 3.0f * inv_p);
        const int s1 = it.subface >= 0 ? it.subface / 3 : (int)(((float)b + 0.5f) * 3.0f * inv_p);
        const int slot = it.subface >= 0 ? 0 : s0 + 3 * s1;
        const double* fc = g_fine + it.fine_offset + slot * arr +
                           frame_vol(fr, -1, 3 * a + 1 - s0 * p, 3 * b + 1 - s1 * p) * U + t.u0 + lane;
        // all 27 loads first (independent, in flight together), then the rounding
        const unsigned long long last = l2_policy_evict_first();
        double gv[3][3][3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int e0 = 0; e0 < 3; ++e0)
#pragma unroll
            for (int e1 = 0; e1 < 3; ++e1)
              gv[ii][e0][e1] = ld_hint(fc - min(ii, k - 1) * gs_n + (e0 - 1) * gs_a + (e1 - 1) * gs_b, last);
        long long n[3][3][3];  // [ii][e0 + 1][e1 + 1]
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int e0 = 0; e0 < 3; ++e0)
#pragma unroll
            for (int e1 = 0; e1 < 3; ++e1) n[ii][e0][e1] = ii < k ? quantize_pow2(gv[ii][e0][e1], s) : 0;
        auto add = [&](int j, int aa, int bb, long long v) {
          atomicAdd((unsigned long long*)&acc[(((j - rlo) * p + bb) * p + aa) * 32 + lane], (unsigned long long)v);
        };
        if (m == 1) {
          dlinear_fixed_adjoint([&](int ii, int e0, int e1) { return n[ii][e0 + 1][e1 + 1]; }, add, k, p, a, b);
          continue;
        }
        // moments: along t1, then t0, then the normal (child ii sits at
        // normal offset +1, 0, -1 for ii = 0, 1, 2)
        Mom3 R[3][3];  // [ii][e0] -> t1 moments
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int e0 = 0; e0 < 3; ++e0) R[ii][e0] = mom3(n[ii][e0][0], n[ii][e0][1], n[ii][e0][2]);
        Mom3 S[3][3];  // [ii][class of z] -> t0 moments
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int zc = 0; zc < 3; ++zc) {
            auto pk = [&](const Mom3& v) { return zc == 0 ? v.s0 : (zc == 1 ? v.od : v.ev); };
            S[ii][zc] = mom3(pk(R[ii][0]), pk(R[ii][1]), pk(R[ii][2]));
          }
        auto gmom = [&](int x, int y, int z) -> long long {
          const int zc = z == 0 ? 0 : ((z & 1) ? 1 : 2);
          const int yc = y == 0 ? 0 : ((y & 1) ? 1 : 2);
          auto pk = [&](const Mom3& v) { return yc == 0 ? v.s0 : (yc == 1 ? v.od : v.ev); };
          // normal values at offsets -1, 0, +1 are children ii = 2, 1, 0
          const Mom3 T = mom3(pk(S[2][zc]), pk(S[1][zc]), pk(S[0][zc]));
          return mom_pick(T, x);
        };
        if (m == 3) taylor_fixed_adjoint<3>(gmom, add, k, p, a, b);
        else taylor_fixed_adjoint<2>(gmom, add, k, p, a, b);
      }
    }
  }
  __syncthreads();
  // every value of the coarse face array (chunk of unknowns)
  const uint32_t ovf_hi = finite ? 0x7ff00000u : 0x7ff80000u;
  const int sh = finite ? s : -4000;
  if (lane < nu) {
    // a warp takes one row (signed layer j, bb) of p volumes along t0 at a time
    const int nrow = 2 * k * p;
    int j = -k, bb = warp;
    while (bb >= p) { bb -= p; ++j; }
    for (int row = warp; row < nrow; row += nw) {
      double* dst = g_coarse + first.coarse_offset + frame_vol(fr, j, 0, bb) * U + t.u0 + lane;
      const bool in = j >= rlo && j <= rhi;
      const long long* src = acc + (((j - rlo) * p + bb) * p) * 32 + lane;
      for (int aa = 0; aa < p; ++aa) dst[aa * gs_a] = in ? adj_to_f64(src[aa * 32], sh, ovf_hi) : 0.0;
      bb += nw;
      while (bb >= p) { bb -= p; ++j; }
    }
  }
}

// g_fine = R^T g_coarse for the Taylor items (finite differences or least
// squares) with p a multiple of 3: one CTA per fine face array, which it
// writes whole.  First the array is zeroed with flat 16-byte stores (memory
// order, full sectors); then, after a barrier, the derivative window of each
// coincident column (fine local indices q0, q1 = 1 mod 3) is written: fine
// layer s + i gets [s + i == 1] g_0 + sum_{j >= 1} W_j[i] g_j from coarse halo
// column ((q0 + s0 p - 1) / 3, (q1 + s1 p - 1) / 3); one warp per window
// volume, lane = unknown.
__global__ void __launch_bounds__(256) restrict_adjoint_taylor_kernel(const amr_transfer_item* __restrict__ items,
                                                                      const Tile* __restrict__ tiles, int U,
                                                                      const double* __restrict__ g_coarse,
                                                                      double* __restrict__ g_fine) {
  const Tile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  const int64_t arr = fr.vols * U;
  double* fa = g_fine + it.fine_offset + (int64_t)t.slot * arr;
  {
    const int head = (reinterpret_cast<uintptr_t>(fa) & 15) ? 1 : 0;  // fa is 8-byte aligned
    const int64_t n2 = (arr - head) / 2;
    double2* v2 = reinterpret_cast<double2*>(fa + head);
    for (int64_t q = threadIdx.x; q < n2; q += blockDim.x) v2[q] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0 && head) fa[0] = 0.0;
    if (threadIdx.x == 0 && head + 2 * n2 < arr) fa[arr - 1] = 0.0;
  }
  __syncthreads();
  const int s0 = t.sub % 3, s1 = t.sub / 3;
  const int gs_n = (int)fr.s_n * U;
  int s, L;
  stencil_window(k - 1, -k, k - 1, pure_exactness(m), s, L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nc = p / 3;  // coincident columns per axis
  for (int w = warp; w < nc * nc * L; w += nw) {
    const int i = w % L, cc = w / L;
    const int q0 = 3 * (cc % nc) + 1, q1 = 3 * (cc / nc) + 1;
    const double* gc = g_coarse + it.coarse_offset + frame_vol(fr, 0, (q0 + s0 * p - 1) / 3, (q1 + s1 * p - 1) / 3) * U;
    double* dst = fa + frame_vol(fr, s + i, q0, q1) * U;
    for (int u = lane; u < U; u += 32) {
      double val = s + i == 1 ? __ldg(gc + u) : 0.0;  // coarse layer 0 injects fine layer 1
      for (int jj = 1; jj < k; ++jj) val = fma(c_rw[rw_index(m, k, jj, it.scheme) + i], __ldg(gc + jj * gs_n + u), val);
      dst[u] = val;
    }
  }
}

}  // namespace amr
