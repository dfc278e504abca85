// Exact fixed-point interpolation (AMR_PREC_FIXED).
//
// The Taylor operators of Sec. 3 and the d-linear operator of Sec. 2 are
// linear maps with rational weights: in units of the fine spacing every
// Taylor coefficient is (integer combination of stencil values) / G, with
// G = 648 (Taylor-3), 36 (Taylor-2) or 27 (d-linear).  This path makes the
// whole evaluation exact integer arithmetic:
//   * each staged coarse value x of unknown u is quantized once to an integer
//     n = round(x / q) on the grid q = 3^g3 2^-s (G = 2^g2 3^g3), with s
//     chosen per tile and unknown so that |n| < 2^47 over the tile's stencil
//     region (one float64 FMA against a magic constant per staged value);
//   * the stencil differences n_j - n_c, the derivative numerators, the
//     scaling to the common denominator and the even/odd evaluation of the
//     27 children run in int64 and are exact: the largest intermediate is
//     below 2^14 times the largest difference, so nothing overflows;
//   * a child is T q / G = T 2^-(s + g2) with T = G n_c + S exact; T is
//     rebuilt as float64 by integer normalisation and rounded once.
// The only error is the quantization of the inputs, |x - n q| <= q / 2, i.e.
// at most about 2^-47 of the largest magnitude in the region, propagated
// through the operator (row sums of |weights| below 10): about 1e-13
// normwise, the precision of float64 arithmetic.  No float32 is involved.
#pragma once
#include "transfer_kernels.cuh"

namespace amr {

constexpr int kFixedBits = 47;             // staged values satisfy |n| < 2^47
// CTA size of the fixed-point kernel; two CTAs per SM (a whole-face region
// of 32 unknowns fills ~104 KB of shared memory), so it also sets the
// registers per thread (65536 / (2 x threads)).  Build option.
#ifndef AMR_FIXED_THREADS
#define AMR_FIXED_THREADS 256
#endif
constexpr int kMaxFixedThreads = AMR_FIXED_THREADS;
constexpr long long kMagicBits = 0x4338000000000000LL;  // bit pattern of 1.5 * 2^52

__constant__ int32_t c_fxw[WT_SIZE];  // integer stencil numerators (Tables::fxw)

// Common denominator G = 2^g2 3^g3 of the Taylor coefficients (fine units) of
// order m, and fl3 = floor(g3 log2 3).
struct FixedScale {
  int g2, g3, G, fl3;
  double inv3;  // 3^-g3
};
__device__ __forceinline__ FixedScale fixed_scale(int m) {
  FixedScale f;
  if (m == 3) { f.g2 = 3; f.g3 = 4; f.G = 648; f.fl3 = 6; f.inv3 = 1.0 / 81.0; }
  else if (m == 2) { f.g2 = 2; f.g3 = 2; f.G = 36; f.fl3 = 3; f.inv3 = 1.0 / 9.0; }
  else { f.g2 = 0; f.g3 = 3; f.G = 27; f.fl3 = 4; f.inv3 = 1.0 / 27.0; }
  return f;
}

// T * 2^-sh as float64, rounded to nearest (ties away from zero), by integer
// normalisation (no float64 instruction).  |T| < 2^63.  A result below the
// float64 normal range becomes +0; above it, the bit pattern ovf_hi:0
// (signed infinity, or a NaN for a tile whose region held one).
__device__ __forceinline__ double fixed_to_f64(long long T, int sh, uint32_t ovf_hi) {
  const unsigned long long sg = (unsigned long long)(T >> 63);
  unsigned long long m = ((unsigned long long)T ^ sg) - sg;
  const int lz = __clzll(m);
  m <<= (lz & 63);
  m = (m >> 1) + 0x200ull;  // leading one at bit 62; half an ulp of the 53-bit result
  const unsigned long long mant = m >> 10;  // 2^52 + fraction, or 2^53 when rounding carried
  // biased exponent - 1: the leading one of mant adds the missing 1 (and a
  // rounding carry into bit 53 moves the exponent up by one, as it must)
  const int e = 1085 - lz - sh;
  uint32_t hi = (uint32_t)(mant >> 32) + ((uint32_t)e << 20);
  uint32_t lo = (uint32_t)mant;
  hi |= (uint32_t)sg & 0x80000000u;
  if (e < 0 || lz == 64) { hi = 0u; lo = 0u; }
  if (e >= 2046) { hi = ovf_hi | ((uint32_t)sg & 0x80000000u); lo = 0u; }
  return __hiloint2double((int)hi, (int)lo);
}

// The same value through the float64 unit: one hardware int64 -> float64
// conversion (rounded to nearest even), then the scaling by 2^-sh applied to
// the exponent field with integer operations.  Same range handling.
__device__ __forceinline__ double fixed_to_f64_unit(long long T, int sh, uint32_t ovf_hi) {
  const double d = __ll2double_rn(T);
  uint32_t hi = (uint32_t)__double2hiint(d);
  uint32_t lo = (uint32_t)__double2loint(d);
  const uint32_t sign = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);  // 0 only for T == 0
  const int En = E - sh;
  hi -= (uint32_t)sh << 20;
  if (E == 0 || En <= 0) { hi = 0u; lo = 0u; }
  if (En >= 2047) { hi = ovf_hi | sign; lo = 0u; }
  return __hiloint2double((int)hi, (int)lo);
}

// 3-point first-derivative numerator (denominator 2) at window position pos:
// the centred difference plus 2 (pos - 1) times the second difference
// (pos 0: -3 x0 + 4 x1 - x2, pos 2: x0 - 4 x1 + 3 x2), branch free.
__device__ __forceinline__ long long fx_r1_3(long long x0, long long x1, long long x2, int pos) {
  return (x2 - x0) + (long long)(2 * (pos - 1)) * (x0 - 2 * x1 + x2);
}
// 3-point second-derivative numerator (lambda / 2!, denominator 2): any position.
__device__ __forceinline__ long long fx_r2_3(long long x0, long long x1, long long x2) { return x0 - 2 * x1 + x2; }

// Pure-line Taylor-coefficient numerators of one axis, already scaled to the
// common denominator, from the values y(i) = n(window point i) - n_c of the
// window read in the direction that puts the centre at position pp <= 2
// (positions 3 and 4 are mirror images of 1 and 0: the caller reads the
// window backwards and negates the odd derivatives).
// Taylor-3, 5-point windows, numerators over 12, 24, 12, scaled by 18, 3, 2.
template <typename Y>
__device__ __forceinline__ void fx_pure5(const Y& y, int pp, long long& r1, long long& r2, long long& r3) {
  if (pp == 2) {  // centred: symmetric and antisymmetric parts
    const long long xm2 = y(0), xm1 = y(1), xp1 = y(3), xp2 = y(4);
    const long long a1 = xp1 - xm1, a2 = xp2 - xm2, s1 = xp1 + xm1, s2 = xp2 + xm2;
    r1 = 144 * a1 - 18 * a2;  // 18 (8 a1 - a2)
    r2 = 48 * s1 - 3 * s2;    // 3 (16 s1 - s2)
    r3 = 2 * a2 - 4 * a1;     // 2 (a2 - 2 a1)
  } else if (pp == 1) {  // (-3, -10, 18, -6, 1), (11, -20, 6, 4, -1), (-3, 10, -12, 6, -1)
    const long long y0 = y(0), y2 = y(2), y3 = y(3), y4 = y(4);
    r1 = 18 * (18 * y2 - 3 * y0 - 6 * y3 + y4);
    r2 = 3 * (11 * y0 + 6 * y2 + 4 * y3 - y4);
    r3 = 2 * (6 * y3 - 3 * y0 - 12 * y2 - y4);
  } else {  // pp == 0: (-25, 48, -36, 16, -3), (35, -104, 114, -56, 11), (-5, 18, -24, 14, -3)
    const long long y1 = y(1), y2 = y(2), y3 = y(3), y4 = y(4);
    r1 = 18 * (48 * y1 - 36 * y2 + 16 * y3 - 3 * y4);
    r2 = 3 * (114 * y2 - 104 * y1 - 56 * y3 + 11 * y4);
    r3 = 2 * (18 * y1 - 24 * y2 + 14 * y3 - 3 * y4);
  }
}

// ---------------------------------------------------------------------------
// Taylor-m (m = 2, 3) interpolation of one coarse centre (layer cl, a, b) and
// one unknown in exact integers.  D(j, a', b') returns n(j, a', b') - n_c.
// emit(ii, e0, e1, S) receives S = G (child - centre) / q for the child ii < kk
// below the centre and tangential offsets e0, e1 (as taylor_interp_core).
// ---------------------------------------------------------------------------
template <int M, typename Diff, typename Emit>
__device__ __forceinline__ void taylor_fixed_core(const Diff& D, const Emit& emit, int k, int p, int a, int b,
                                                  int cl = -1, int kk = 3) {
  const int c[3] = {cl, a, b};
  const int lo[3] = {-k, 0, 0};
  const int hi[3] = {k - 1, p - 1, p - 1};
  int ps[3], pl[3], ms[3], ml[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    stencil_window(c[d], lo[d], hi[d], pure_exactness(M), ps[d], pl[d]);
    stencil_window(c[d], lo[d], hi[d], mixed_exactness(M), ms[d], ml[d]);
  }
  long long C[M + 1][M + 1][M + 1];
#pragma unroll
  for (int x = 0; x <= M; ++x)
#pragma unroll
    for (int y = 0; y <= M; ++y)
#pragma unroll
      for (int z = 0; z <= M; ++z) C[x][y][z] = 0;

  // pure derivatives along each axis, scaled to the common denominator:
  // Taylor-3 (windows of 4 or 5, numerators over 12, 24, 12): M_r = 18, 3, 2;
  // Taylor-2 (windows of 3, numerators over 2): M_r = 6, 2
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int pos = c[d] - ps[d], L = pl[d];
    auto at = [&](int i) -> long long {
      int x[3] = {c[0], c[1], c[2]};
      x[d] = ps[d] + i;
      return D(x[0], x[1], x[2]);
    };
    long long r1, r2, r3 = 0;
    if (M == 3 && L == 5) {
      const bool back = pos > 2;  // mirror image of position 4 - pos
      auto y = [&](int i) -> long long { return at(back ? 4 - i : i); };
      fx_pure5(y, back ? 4 - pos : pos, r1, r2, r3);
      if (back) {
        r1 = -r1;
        r3 = -r3;
      }
    } else if (M == 3 && L == 4 && pos == 1) {  // the normal line at k = 2
      const long long y0 = at(0), y2 = at(2), y3 = at(3);
      r1 = 18 * (12 * y2 - 4 * y0 - 2 * y3);
      r2 = 3 * (12 * y0 + 12 * y2);
      r3 = 2 * (2 * y3 - 2 * y0 - 6 * y2);
    } else if (M == 2 && L == 3) {
      const long long x0 = at(0), x1 = at(1), x2 = at(2);  // the centre's own value is 0
      r1 = 6 * fx_r1_3(x0, x1, x2, pos);
      r2 = 2 * fx_r2_3(x0, x1, x2);
    } else {  // any other window (short tangential ranges): numerators from the table
      const int32_t* w = c_fxw + wt_offset(L) + pos * 3 * L;
      long long acc[3] = {0, 0, 0};
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        if (i < L && i != pos) {
          const long long v = at(i);
#pragma unroll
          for (int r = 0; r < M; ++r) acc[r] += (long long)w[r * L + i] * v;
        }
      }
      if (M == 3) {
        r1 = 18 * acc[0];
        r2 = 3 * acc[1];
        r3 = 2 * acc[2];
      } else {
        r1 = 6 * acc[0];
        r2 = 2 * acc[1];
      }
    }
    if (d == 0) { C[1][0][0] = r1; C[2][0][0] = r2; if (M == 3) C[3][0][0] = r3; }
    if (d == 1) { C[0][1][0] = r1; C[0][2][0] = r2; if (M == 3) C[0][3][0] = r3; }
    if (d == 2) { C[0][0][1] = r1; C[0][0][2] = r2; if (M == 3) C[0][0][3] = r3; }
  }

  // Mixed derivatives from the 3x3x3 box of the 3-point windows (normal
  // window always centred on the centre's layer), collapsed along the normal, then t0,
  // then t1, each box value read once; numerators over 2 per differentiated
  // axis.  Taylor-2 needs only the three planes through the centre.
  {
    const int sa = c[1] - ms[1], sb = c[2] - ms[2];
    long long P11[3], P01[3], P10[3], P20[3], P02[3], P21[3], P12[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      long long S1[3], S2[3], X1[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        X1[j] = D(ms[0] + 1, ms[1] + j, ms[2] + q);  // layer -1: the centre's own plane
        if (M == 3 || q == sb || j == sa) {
          const long long x0 = D(ms[0], ms[1] + j, ms[2] + q);
          const long long x2 = D(ms[0] + 2, ms[1] + j, ms[2] + q);
          S1[j] = x2 - x0;
          S2[j] = x0 - 2 * X1[j] + x2;
        } else {
          S1[j] = S2[j] = 0;
        }
      }
      P11[q] = fx_r1_3(S1[0], S1[1], S1[2], sa);
      P01[q] = fx_r1_3(X1[0], X1[1], X1[2], sa);
      P10[q] = sa == 0 ? S1[0] : (sa == 1 ? S1[1] : S1[2]);
      if (M == 3) {
        P20[q] = sa == 0 ? S2[0] : (sa == 1 ? S2[1] : S2[2]);
        P02[q] = fx_r2_3(X1[0], X1[1], X1[2]);
        P21[q] = fx_r1_3(S2[0], S2[1], S2[2], sa);
        P12[q] = fx_r2_3(S1[0], S1[1], S1[2]);
      }
    }
    auto at3 = [&](const long long* v) -> long long { return sb == 0 ? v[0] : (sb == 1 ? v[1] : v[2]); };
    const long long m110 = at3(P11);
    const long long m101 = fx_r1_3(P10[0], P10[1], P10[2], sb);
    const long long m011 = fx_r1_3(P01[0], P01[1], P01[2], sb);
    if (M == 3) {
      // scaling to G = 648: (1,1) 648 / (4 * 9) = 18, (2,1) 648 / (4 * 27) = 6,
      // (1,1,1) 648 / (8 * 27) = 3
      C[1][1][0] = 18 * m110; C[1][0][1] = 18 * m101; C[0][1][1] = 18 * m011;
      C[2][1][0] = 6 * at3(P21);
      C[1][2][0] = 6 * at3(P12);
      C[2][0][1] = 6 * fx_r1_3(P20[0], P20[1], P20[2], sb);
      C[1][0][2] = 6 * fx_r2_3(P10[0], P10[1], P10[2]);
      C[0][2][1] = 6 * fx_r1_3(P02[0], P02[1], P02[2], sb);
      C[0][1][2] = 6 * fx_r2_3(P01[0], P01[1], P01[2]);
      C[1][1][1] = 3 * fx_r1_3(P11[0], P11[1], P11[2], sb);
    } else {
      // G = 36: (1,1) 36 / (4 * 9) = 1
      C[1][1][0] = m110; C[1][0][1] = m101; C[0][1][1] = m011;
    }
  }
  taylor_children<M, long long>(C, emit, kk < k ? kk : k);
}

// d-linear interpolation of one coarse centre in exact integers (G = 27:
// each 1-D lerp has weights in thirds).  D and emit as above (the centre's
// own difference is 0).
template <typename Diff, typename Emit>
__device__ __forceinline__ void dlinear_fixed_core(const Diff& D, const Emit& emit, int k, int p, int a, int b,
                                                   int cl = -1, int kk = 3) {
  if (kk > k) kk = k;
  const bool alo = a == 0, ahi = a == p - 1, blo = b == 0, bhi = b == p - 1;
  const int aidx[3] = {alo ? a : a - 1, a, ahi ? a : a + 1};
  const int bidx[3] = {blo ? b : b - 1, b, bhi ? b : b + 1};
  long long N[3][3][3];  // 3 x the normal lerp: [child normal ii][da][db]
#pragma unroll
  for (int da = 0; da < 3; ++da)
#pragma unroll
    for (int db = 0; db < 3; ++db) {
      const long long v1 = D(cl, aidx[da], bidx[db]);
      const long long v0 = D(cl + 1, aidx[da], bidx[db]);
      N[0][da][db] = 2 * v1 + v0;  // child above: v1 + (v0 - v1) / 3
      N[1][da][db] = 3 * v1;       // child coincident with coarse layer cl
      N[2][da][db] = 3 * v1;
      if (kk >= 3) N[2][da][db] = 2 * v1 + D(cl - 1, aidx[da], bidx[db]);  // child below
    }
  // 3 x the 1-D lerp to offsets -1, 0, +1 (linear extrapolation at an edge)
  auto lerp3 = [](long long xm, long long x0, long long xp, bool le, bool he, long long& rm, long long& rz,
                  long long& rp) {
    rz = 3 * x0;
    rm = le ? 4 * x0 - xp : 2 * x0 + xm;
    rp = he ? 4 * x0 - xm : 2 * x0 + xp;
  };
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) {
    if (ii >= kk) break;
    long long Am[3], Az[3], Ap[3];
#pragma unroll
    for (int db = 0; db < 3; ++db) lerp3(N[ii][0][db], N[ii][1][db], N[ii][2][db], alo, ahi, Am[db], Az[db], Ap[db]);
#pragma unroll
    for (int e0 = -1; e0 <= 1; ++e0) {
      const long long* A = e0 < 0 ? Am : (e0 == 0 ? Az : Ap);
      long long rm, rz, rp;
      lerp3(A[0], A[1], A[2], blo, bhi, rm, rz, rp);
      emit(ii, e0, -1, rm);
      emit(ii, e0, 0, rz);
      emit(ii, e0, 1, rp);
    }
  }
}

// ---------------------------------------------------------------------------
// Interpolation kernel, fixed point.  One CTA per tile (<= 32 unknowns), one
// warp per coarse centre with lane = unknown.  Phase 1 stages the region's
// float64 values in shared memory and finds, per unknown, the largest
// exponent; phase 2 quantizes them in place; phase 3 evaluates the children.
// ---------------------------------------------------------------------------
// CVT: which children are converted on the float64 unit (fixed_to_f64_unit)
// instead of by integer normalisation (fixed_to_f64), balancing the two
// pipes: 0 none, 1 e0 <= 0 and e1 <= 0 (4/9), 2 e1 <= 0 (2/3), 3 all but
// e0 = e1 = +1 (8/9).  The autotuner picks it (tuning field interp_addback).
template <bool CUT, int CVT = 0>
__global__ void __launch_bounds__(kMaxFixedThreads, 2)
    interp_fixed_kernel(const amr_transfer_item* __restrict__ items, const Tile* __restrict__ tiles, int U,
                        const double* __restrict__ coarse, double* __restrict__ fine) {
  extern __shared__ double smem_raw[];
  long long* sm = reinterpret_cast<long long*>(smem_raw);
  __shared__ int s_emax[32];
  const Tile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  IRange rn, ra, rb;
  interp_region(p, k, m, t.a0, t.na, t.b0, t.nb, rn, ra, rb);
  const int NA = ra.hi - ra.lo + 1, NB = rb.hi - rb.lo + 1, NJ = rn.hi - rn.lo + 1;
  const int nu = t.nu;  // <= 32
  const int gs_n = (int)fr.s_n * U, gs_a = (int)fr.s_t0 * U, gs_b = (int)fr.s_t1 * U;
  const double* cb = coarse + it.coarse_offset + t.u0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int npts = NJ * NB * NA;
  // the host sizes the launch for the largest region (32 slots per volume);
  // a tile whose region would not fit is left unwritten rather than staged
  // out of bounds
  uint32_t dyn_smem;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
  if ((uint32_t)npts * 32u * 8u > dyn_smem || nu > 32) return;
  if (threadIdx.x < 32) s_emax[threadIdx.x] = 0;
  __syncthreads();
  // phase 1: warp w stages points w, w + nw, ...; lane = unknown
  if (lane < nu) {
    const double* g0 = cb + frame_vol(fr, rn.lo, ra.lo, rb.lo) * U + lane;
    Counter4 c;
    c.init(warp, nw, 1, NA, NB);
    int emax = 0;
    constexpr int STAGE = 8;
    for (int p0 = warp; p0 < npts; p0 += STAGE * nw) {
      double v[STAGE];
#pragma unroll
      for (int q = 0; q < STAGE; ++q) {
        if (p0 + q * nw < npts) v[q] = __ldg(g0 + c.z * gs_n + c.y * gs_b + c.x * gs_a);
        c.advance(1, NA, NB);
      }
#pragma unroll
      for (int q = 0; q < STAGE; ++q) {
        if (p0 + q * nw < npts) {
          const long long bits = __double_as_longlong(v[q]);
          sm[(p0 + q * nw) * 32 + lane] = bits;
          emax = max(emax, (int)((bits >> 52) & 0x7ff));
        }
      }
    }
    atomicMax(&s_emax[lane], emax);
  }
  __syncthreads();
  // per-unknown grid: |x| < 2^(E - 1022) for the largest biased exponent E of
  // the region; n = round(x 2^s / 3^g3) with s = 47 - e_m + fl3 keeps
  // |n| < 2^47.  Regions whose largest magnitude is below 2^-960 use the
  // grid of 2^-960 (a finer grid would overflow the scale factor).
  const FixedScale fs = fixed_scale(m);
  const int E = lane < nu ? s_emax[lane] : 0;
  const bool finite = E < 2047;
  const int e_m = max(E, 62) - 1022;
  const int s = kFixedBits - e_m + fs.fl3;
  const double qinv = __longlong_as_double(__double_as_longlong(fs.inv3) + ((long long)s << 52));
  // phase 2: quantize in place (one float64 FMA each)
  if (lane < nu) {
    for (int pt = warp; pt < npts; pt += nw) {
      const double x = __longlong_as_double(sm[pt * 32 + lane]);
      const double tq = __fma_rn(x, qinv, 6755399441055744.0);  // + 1.5 * 2^52
      sm[pt * 32 + lane] = finite ? __double_as_longlong(tq) - kMagicBits : 0;
    }
  }
  __syncthreads();
  // children are T 2^-(s + g2) with T = G n_c + S; a non-finite region makes
  // every computed child NaN (shift forced past the overflow threshold)
  const int sh = finite ? s + fs.g2 : -4000;
  const uint32_t ovf_hi = finite ? 0x7ff00000u : 0x7ff80000u;
  const int64_t arr = fr.vols * U;
  const float inv_p = 1.0f / (float)p;
  // region point (j, b, a) of unknown u at ((j * NB + b) * NA + a) * 32 + u:
  // neighbours along t0 are compile-time offsets
  constexpr int SA = 32;
  const int SB = NA * 32, SJ = NB * NA * 32;
  const int ntask = t.na * t.nb * centre_layers(k);  // centres (a, b) of each centre layer
  Counter4 c;
  c.init(warp, nw, 1, t.na, t.nb);
  for (int e = lane < nu ? warp : ntask; e < ntask; e += nw, c.advance(1, t.na, t.nb)) {
    const int u = lane, a = t.a0 + c.x, b = t.b0 + c.y;
    const int cl = -1 - c.z, kk = child_layers(k, c.z);  // centre layer and its child layers
    ChildMap cm;
    CutAxis ca, cbx;
    if constexpr (CUT) {
      int s0 = t.sub % 3, s1 = t.sub / 3;
      cm.slot = t.slot;
      if (t.sub < 0) {
        s0 = (int)(__fmaf_rn((float)a, 3.f, 1.5f) * inv_p);
        s1 = (int)(__fmaf_rn((float)b, 3.f, 1.5f) * inv_p);
        cm.slot = s0 + 3 * s1;
      }
      cm.q0_off = 1 - s0 * p;
      cm.q1_off = 1 - s1 * p;
      ca = cut_axis(t.sub < 0, 3 * a + cm.q0_off, p, gs_a, arr);
      cbx = cut_axis(t.sub < 0, 3 * b + cm.q1_off, p, gs_b, 3 * arr);
    } else {
      cm = child_map(t, p, a, b);
    }
    double* fc = fine + it.fine_offset + (int64_t)cm.slot * arr +
                 frame_vol(fr, cl - 2 * c.z, 3 * a + cm.q0_off, 3 * b + cm.q1_off) * U + t.u0 + u;
    const int ic = (((cl - rn.lo) * NB + (b - rb.lo)) * NA + (a - ra.lo)) * 32 + u;
    const long long nc = sm[ic];
    const long long Gnc = (long long)fs.G * nc;
    const double base = __ldg(cb + frame_vol(fr, cl, a, b) * U + u);
    auto D = [&](int j, int aa, int bb) -> long long {
      return sm[ic + (j - cl) * SJ + (bb - b) * SB + (aa - a) * SA] - nc;
    };
    auto emit = [&](int ii, int e0, int e1, long long S) {
      double v;
      if (ii == 1 && e0 == 0 && e1 == 0) v = base;
      else if ((CVT == 1 && e0 <= 0 && e1 <= 0) || (CVT == 2 && e1 <= 0) || (CVT == 3 && (e0 < 1 || e1 < 1)))
        v = fixed_to_f64_unit(Gnc + S, sh, ovf_hi);
      else v = fixed_to_f64(Gnc + S, sh, ovf_hi);
      if constexpr (CUT) {
        if (cut_valid(ca, e0) && cut_valid(cbx, e1)) fc[-ii * gs_n + cut_off(ca, e0) + cut_off(cbx, e1)] = v;
      } else {
        fc[-ii * gs_n + e0 * gs_a + e1 * gs_b] = v;
      }
    };
    if (m == 3) taylor_fixed_core<3>(D, emit, k, p, a, b, cl, kk);
    else if (m == 2) taylor_fixed_core<2>(D, emit, k, p, a, b, cl, kk);
    else dlinear_fixed_core(D, emit, k, p, a, b, cl, kk);
  }
}

}  // namespace amr
