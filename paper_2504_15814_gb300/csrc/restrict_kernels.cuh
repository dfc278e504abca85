// sm_103a restriction kernel of the coarse<->fine transfer (coarse halo
// volumes = R fine face arrays; paper Sec. 2, Sec. 3): one thread per
// (coarse halo column, unknown) reads the coincident fine normal line, no
// staging.  Taylor items: injection plus extrapolation with combined
// weights, in float64, float-pair (split plans) or float64 and exact integer
// columns side by side (fixed-point plans); d-linear items: tangential
// average and normal least-squares line.
#pragma once
#include "transfer_kernels.cuh"

namespace amr {

__constant__ int32_t c_rwx[RW_SIZE];         // integer restriction weights (Tables::rwx)
__constant__ int32_t c_rw_den[RW_SIZE / 5];  // their row denominators 2^a 3^b as a | b << 4
__constant__ int32_t c_lsx[LS_SIZE];         // d-linear line weights / 9 as integers (Tables::lsx)
__constant__ int32_t c_ls_den[kMaxOverlap * kMaxOverlap];  // a | b << 4 | usable << 8 per (k, j)

// ---------------------------------------------------------------------------
// Restriction tasks: one coarse halo column (a, b), one unknown.  F(i, da, db)
// reads the fine volume at signed layer i, tangential offset (da, db) from the
// fine column coincident with the coarse centre; C(j, v) writes coarse halo
// layer j.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double pick5(const double* v, int idx) {
  double r = v[0];
#pragma unroll
  for (int i = 1; i < 5; ++i) r = (i == idx) ? v[i] : r;
  return r;
}

// Taylor restriction in split mode, window values v[0..L) already loaded
// (expansion value v[pos]): exact float-pair differences to the expansion
// value, formed once per column; per extrapolated layer j >= j0 a float-pair
// weighted sum; each output rebuilt as float64 without float64 instructions.
template <typename Store>
__device__ __forceinline__ void taylor_extrapolate_split(const double* v, int L, int pos, int m, int k, int j0,
                                                         int j1, int scheme, const Store& store) {
  const F2 b = split_f64(pick5(v, pos));
  float dh[5], dl[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    dh[i] = 0.f;
    dl[i] = 0.f;
    if (i < L && i != pos) {
      const F2 x = split_f64(v[i]);
      float e;
      dh[i] = two_sum(x.hi, -b.hi, e);
      dl[i] = __fadd_rn(e, __fsub_rn(x.lo, b.lo));
    }
  }
  for (int j = j0; j < k && j < j1; ++j) {
    const int w0 = rw_index(m, k, j, scheme);
    float ah = 0.f, al = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float wh = c_rw_hi[w0 + i], wl = c_rw_lo[w0 + i];
      const float pr = __fmul_rn(wh, dh[i]);
      float pe = __fmaf_rn(wh, dh[i], -pr);  // exact product error
      pe = __fmaf_rn(wh, dl[i], pe);
      pe = __fmaf_rn(wl, dh[i], pe);
      float t;
      ah = two_sum(ah, pr, t);
      al = __fadd_rn(al, __fadd_rn(t, pe));
    }
    float e1, e2;
    const float s1 = two_sum(b.hi, ah, e1);
    const float tt = __fadd_rn(__fadd_rn(e1, b.lo), al);
    const float s2 = fast_two_sum(s1, tt, e2);
    store(j, pair_to_f64(s2, e2));
  }
}

// d-linear, float64: tangential 3x3 average per fine layer, least-squares
// line along the normal.  All loads are issued before the arithmetic.
template <typename Fine, typename Coarse>
__device__ __forceinline__ void dlinear_restrict_f64(const Fine& F, const Coarse& C, int k) {
  const int nl = k == 1 ? 2 : k;
  double avg[kMaxOverlap] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int sl = 0; sl < kMaxOverlap; ++sl) {
    if (sl < nl) {
      double v[9];  // one fine layer: all 9 loads before the sum
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = F(k == 1 ? sl - 1 : sl, q % 3 - 1, q / 3 - 1);
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) acc += v[q];
      avg[sl] = acc * (1.0 / 9.0);
    }
  }
  for (int j = 0; j < k; ++j) {
    double r = 0.0;
#pragma unroll
    for (int sl = 0; sl < kMaxOverlap; ++sl)
      if (sl < nl) r += c_ls[ls_index(k, j, sl)] * avg[sl];
    C(j, r);
  }
}

// d-linear, split: the same weights applied in float32 to exact float-pair
// differences against the column's value in fine layer 0 (weights <= 10/3).
template <typename Fine, typename Coarse>
__device__ __forceinline__ void dlinear_restrict_split(const Fine& F, const Coarse& C, int k) {
  const int nl = k == 1 ? 2 : k;
  const F2 r = split_f64(F(0, 0, 0));  // fine layer 0, centre column
  float avg[kMaxOverlap] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int sl = 0; sl < kMaxOverlap; ++sl) {
    if (sl < nl) {
      double v[9];  // one fine layer: all 9 loads before the arithmetic
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = F(k == 1 ? sl - 1 : sl, q % 3 - 1, q / 3 - 1);
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const F2 x = split_f64(v[q]);
        acc += __fadd_rn(__fsub_rn(x.hi, r.hi), __fsub_rn(x.lo, r.lo));
      }
      avg[sl] = acc * (1.0f / 9.0f);
    }
  }
  for (int j = 0; j < k; ++j) {
    float w = 0.f;
#pragma unroll
    for (int sl = 0; sl < kMaxOverlap; ++sl)
      if (sl < nl) w += c_ls_f[ls_index(k, j, sl)] * avg[sl];
    C(j, add_back(r, w));
  }
}

// ---------------------------------------------------------------------------
// Taylor restriction of one column in integers (fixed-point plans, every
// other column; the float64 unit takes the rest).  The window values
// v[0..L) are rounded once onto the grid 2^-s, s = 1084 - E (E the largest
// biased exponent of the window): |n| < 2^62, rounding error at most 2^-62
// of the window's largest magnitude.  Each n is carried as two signed 31-bit
// halves, so the sums with the integer weights (|W| < 2^15) are exact in two
// int64 accumulators A and B, T = A 2^31 + B.  T 2^-s / D is rounded to
// float64 by integer normalisation: exactly once when |A| < 2^31 (T fits 63
// bits), else after dropping the 17 low bits of B (relative error below
// 2^-44); a row denominator D with a factor 3 adds one float64 multiply by
// 1/3.  Windows with a non-finite value or a largest magnitude outside
// 2^-923 .. 2^977 return false (the caller uses float64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split62(double v, int E, int& nh, int& nl) {
  const long long bits = __double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long M = (unsigned long long)(bits & 0xFFFFFFFFFFFFFll) | (e ? (1ull << 52) : 0ull);
  const int sh = max(e, 1) - E + 9;  // <= 9: |n| = M 2^sh < 2^62
  unsigned long long N;
  if (sh >= 0) N = M << sh;
  else N = -sh <= 54 ? ((M >> (-sh - 1)) + 1) >> 1 : 0ull;  // half away from zero
  const int h = (int)(N >> 31), l = (int)(N & 0x7fffffffull);
  nh = bits < 0 ? -h : h;
  nl = bits < 0 ? -l : l;
}

// T 2^-sh as float64 for 0 < |T| < 2^63 with the result in the normal range:
// integer normalisation, ties away from zero.
__device__ __forceinline__ double scaled_i64_to_f64(long long T, int sh) {
  const unsigned long long sg = (unsigned long long)(T >> 63);
  unsigned long long m = ((unsigned long long)T ^ sg) - sg;
  const int lz = __clzll((long long)m);
  m <<= lz;
  m = (m >> 1) + 0x200ull;           // leading one at bit 62; half an ulp of the 53-bit result
  const unsigned long long mant = m >> 10;  // 2^52 + fraction, or 2^53 after a rounding carry
  const long long e = 1085 - lz - sh;       // biased exponent - 1 (the leading one adds 1)
  return __longlong_as_double((long long)((sg << 63) | (mant + ((unsigned long long)e << 52))));
}

template <typename Store>
__device__ __forceinline__ bool restrict_int_layers(const double* v, int L, int m, int k, const Store& store) {
  int E = 1;
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (i < L) E = max(E, (int)((__double_as_longlong(v[i]) >> 52) & 0x7ff));
  if (E < 100 || E > 2000) return false;
  int nh[5], nl[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    nh[i] = 0;
    nl[i] = 0;
    if (i < L) split62(v[i], E, nh[i], nl[i]);
  }
  const int s = 1084 - E;
  for (int j = 1; j < k; ++j) {
    const int r0 = rw_index(m, k, j);
    long long A = 0, B = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int W = c_rwx[r0 + i];
      A += (long long)W * nh[i];
      B += (long long)W * nl[i];
    }
    const int den = c_rw_den[r0 / 5];
    const bool fits = A < (1ll << 31) && A > -(1ll << 31);
    const long long T = fits ? (A << 31) + B : (A << 14) + (B >> 17);
    double out = T == 0 ? 0.0 : scaled_i64_to_f64(T, s + (den & 15) - (fits ? 0 : 17));
    if (den >> 4) out *= 1.0 / 3.0;
    store(j, out);
  }
  return true;
}

// d-linear restriction of one column in integers (fixed-point plans, half
// the columns): the 9 nl fine values are rounded once onto the grid 2^-s of
// the column's largest magnitude (s = 1084 - E, |n| < 2^62, 31-bit halves as
// above), the 3 x 3 tangential sums of each fine layer are exact, and the
// least-squares line weights / 9 are integers over D = 2^a 3^b, so each halo
// value is one integer normalisation (plus a multiply by 3^-b).  Overlaps 4
// and 5 (denominators with a 5), windows with a non-finite value or a
// largest magnitude outside 2^-923 .. 2^977 return false.
template <typename Fine, typename Coarse>
__device__ __forceinline__ bool dlinear_restrict_int(const Fine& F, const Coarse& C, int k) {
  if (k > 3) return false;
  for (int j = 0; j < k; ++j)
    if (!((c_ls_den[(k - 1) * kMaxOverlap + j] >> 8) & 1)) return false;
  const int nl = k == 1 ? 2 : k;
  int E = 1;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl)
    if (sl < nl) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
        E = max(E, (int)((__double_as_longlong(F(k == 1 ? sl - 1 : sl, q % 3 - 1, q / 3 - 1)) >> 52) & 0x7ff));
    }
  if (E < 100 || E > 2000) return false;
  long long Sh[3] = {0, 0, 0}, Sl[3] = {0, 0, 0};
#pragma unroll
  for (int sl = 0; sl < 3; ++sl)
    if (sl < nl) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        int nh, nlo;
        split62(F(k == 1 ? sl - 1 : sl, q % 3 - 1, q / 3 - 1), E, nh, nlo);
        Sh[sl] += nh;
        Sl[sl] += nlo;
      }
    }
  const int s = 1084 - E;
  for (int j = 0; j < k; ++j) {
    const int den = c_ls_den[(k - 1) * kMaxOverlap + j];
    long long A = 0, B = 0;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl)
      if (sl < nl) {
        const long long W = c_lsx[ls_index(k, j, sl)];
        A += W * Sh[sl];
        B += W * Sl[sl];
      }
    const bool fits = A < (1ll << 31) && A > -(1ll << 31);
    const long long T = fits ? (A << 31) + B : (A << 14) + (B >> 17);
    double out = T == 0 ? 0.0 : scaled_i64_to_f64(T, s + (den & 15) - (fits ? 0 : 17));
    const int b3 = (den >> 4) & 15;
    if (b3) out *= b3 == 1 ? 1.0 / 3.0 : (b3 == 2 ? 1.0 / 9.0 : 1.0 / 27.0);
    C(j, out);
  }
  return true;
}

// Restriction precision modes: float64 throughout (float64 plans); split
// (float64 first extrapolated layer, float-pair second layer, float32
// d-linear averaging on exact float-pair differences); fixed (float64 for
// half the columns, the integer paths above for the other half, float64
// where those do not serve: the two pipes share the work).
constexpr int kRestrictF64 = 0, kRestrictSplit = 1, kRestrictFixed = 2;

template <int RP>
__global__ void __launch_bounds__(256) restrict_kernel(const amr_transfer_item* __restrict__ items,
                                                       const Tile* __restrict__ tiles, int U,
                                                       const double* __restrict__ fine,
                                                       double* __restrict__ coarse) {
  constexpr bool SPLIT = RP == kRestrictSplit;
  const Tile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  const int64_t arr = fr.vols * U;
  const int gs_n = (int)fr.s_n * U, gs_a = (int)fr.s_t0 * U, gs_b = (int)fr.s_t1 * U;
  double* cb = coarse + it.coarse_offset + t.u0;
  const float inv_p = 1.0f / (float)p;
  const int nu = t.nu;
  const int ntask = t.na * t.nb * nu;
  // fine column (layer 0) and coarse halo column (layer 0) of a task; q0, q1:
  // local tangential index of the coincident fine column
  auto columns = [&](const Counter4& c, const double*& fcol, double*& ccol, int& q0, int& q1) {
    const int u = c.u, a = t.a0 + c.x, b = t.b0 + c.y;
    int s0, s1, slot;
    if (t.sub >= 0) {
      s0 = t.sub % 3; s1 = t.sub / 3; slot = t.slot;
    } else {  // whole-face tile: the owner holds fine 3a + 1, and (3a + 3/2) / p
              // is never within 1/(2p) of an integer
      s0 = (int)(__fmaf_rn((float)a, 3.f, 1.5f) * inv_p);
      s1 = (int)(__fmaf_rn((float)b, 3.f, 1.5f) * inv_p);
      slot = s0 + 3 * s1;
    }
    q0 = 3 * a + 1 - s0 * p;
    q1 = 3 * b + 1 - s1 * p;
    fcol = fine + it.fine_offset + (int64_t)slot * arr + t.u0 + frame_vol(fr, 0, q0, q1) * U + u;
    ccol = cb + frame_vol(fr, 0, a, b) * U + u;
  };
  Counter4 c;
  c.init(threadIdx.x, blockDim.x, nu, t.na, t.nb);
  if (m >= 2) {
    // Taylor: the derivative window about fine layer k-1 holds fine layer 1
    // (the injection source); two columns per iteration keep 2 x L loads in
    // flight per thread.
    int s, L;
    stencil_window(k - 1, -k, k - 1, pure_exactness(m), s, L);
    const int pos = k - 1 - s;
    // fine layer 1 lies outside the window only for Taylor-2 with k = 5
    const bool inj_in = 1 - s >= 0 && 1 - s < L;
    constexpr int R = 2;
    for (int e0 = threadIdx.x; e0 < ntask; e0 += R * blockDim.x) {
      double v[R][5], v1[R];
      double* ccol[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const double* fcol;
        int q0, q1;
        columns(c, fcol, ccol[r], q0, q1);
        const bool ok = e0 + r * (int)blockDim.x < ntask;
#pragma unroll
        for (int i = 0; i < 5; ++i) v[r][i] = (ok && i < L) ? __ldg(fcol + (s + i) * gs_n) : 0.0;
        v1[r] = (ok && !inj_in) ? __ldg(fcol + gs_n) : 0.0;
        if (!ok) ccol[r] = nullptr;
        c.advance(nu, t.na, t.nb);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!ccol[r]) continue;
        double* col = ccol[r];
        col[0] = inj_in ? pick5(v[r], 1 - s) : v1[r];  // layer 0 coincides with fine layer 1
        if (RP == kRestrictFixed && r == 1 && it.scheme == 0 &&
            restrict_int_layers(v[r], L, m, k, [&](int j, double out) { col[j * gs_n] = out; }))
          continue;
        if (SPLIT) {
          // layer 1 with float64 combined weights (the float64 unit is idle
          // here); layer 2 in float64 for the first column of the pair and in
          // float-pair arithmetic for the second: the two pipes share the work
          const double* w = c_rw + rw_index(m, k, 1, it.scheme);
          double acc = 0.0;
#pragma unroll
          for (int i = 0; i < 5; ++i) acc = fma(w[i], v[r][i], acc);
          col[gs_n] = acc;
          if (k > 2) {
            if (r == 0) {
              const double* w2 = c_rw + rw_index(m, k, 2, it.scheme);
              double acc2 = 0.0;
#pragma unroll
              for (int i = 0; i < 5; ++i) acc2 = fma(w2[i], v[r][i], acc2);
              col[2 * gs_n] = acc2;
            } else {
              taylor_extrapolate_split(v[r], L, pos, m, k, 2, 3, it.scheme, [&](int j, double out) { col[j * gs_n] = out; });
            }
          }
          for (int j = 3; j < k; ++j) {  // overlaps 4 and 5: deeper layers in float64
            const double* w = c_rw + rw_index(m, k, j, it.scheme);
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < 5; ++i) acc = fma(w[i], v[r][i], acc);
            col[j * gs_n] = acc;
          }
        } else {
          for (int j = 1; j < k; ++j) {
            const double* w = c_rw + rw_index(m, k, j, it.scheme);
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < 5; ++i) acc = fma(w[i], v[r][i], acc);
            col[j * gs_n] = acc;
          }
        }
      }
    }
  } else {
    int round = threadIdx.x >> 5;  // fixed-point plans: warps alternate float64 and integer columns
    for (int e = threadIdx.x; e < ntask; e += blockDim.x, c.advance(nu, t.na, t.nb), ++round) {
      const double* fcol;
      double* ccol;
      int q0, q1;
      columns(c, fcol, ccol, q0, q1);
      // a coarse volume cut by a subface boundary (p not a multiple of 3; the
      // coincident column on the array's edge) is injected along that axis:
      // the three tangential reads collapse onto the coincident column
      const int ga = (q0 == 0 || q0 == p - 1) ? 0 : gs_a, gb = (q1 == 0 || q1 == p - 1) ? 0 : gs_b;
      auto F = [&](int i, int da, int db) -> double { return __ldg(fcol + i * gs_n + da * ga + db * gb); };
      auto C = [&](int j, double v) { ccol[j * gs_n] = v; };
      if (RP == kRestrictFixed && (round & 1) && dlinear_restrict_int(F, C, k)) continue;
      if (SPLIT) dlinear_restrict_split(F, C, k);
      else dlinear_restrict_f64(F, C, k);
    }
  }
}

}  // namespace amr
