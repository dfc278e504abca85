// sm_103a kernels of the coarse<->fine transfer (forward operators).
//
// Work decomposition: one CTA per tile (a rectangle of coarse columns of one
// subface, and a range of unknowns).  Interpolation stages the tile's stencil
// region of the coarse face array in shared memory with coalesced loads along
// the AoS unknown axis, then one thread per (coarse centre, unknown) computes
// the centre's Taylor coefficients (or d-linear partial sums) and writes its
// k * 3 * 3 fine children.  Restriction needs no staging: one thread per
// (coarse halo column, unknown) reads the coincident fine normal line.
//
// Precision: FP64 computes everything in float64.  SPLIT forms the stencil
// differences u_j - u_c in float64, does the interpolation's derivative and
// Taylor arithmetic in float32 and adds the increment back to the float64
// base value; restriction stays float64 (see restrict_kernel).
#pragma once
#include "amr_common.cuh"

namespace amr {

__constant__ double c_wt_interp[WT_SIZE];
__constant__ double c_wt_restrict[WT_SIZE];
__constant__ float c_wt_interp_f[WT_SIZE];
__constant__ float c_wt_restrict_f[WT_SIZE];
__constant__ double c_ls[LS_SIZE];

template <bool SPLIT> struct Arith;
template <> struct Arith<false> {
  using T = double;
  __device__ static const double* wt_interp() { return c_wt_interp; }
  __device__ static const double* wt_restrict() { return c_wt_restrict; }
};
template <> struct Arith<true> {
  using T = float;
  __device__ static const float* wt_interp() { return c_wt_interp_f; }
  __device__ static const float* wt_restrict() { return c_wt_restrict_f; }
};

// Value of the polynomial sum_{i<=deg} c[i] x^i at x in {-1, 0, +1}: returns
// (P(-1), P(0), P(+1)) via even/odd parts.
template <typename T>
struct Tri { T m, z, p; };

// ---------------------------------------------------------------------------
// Taylor-m interpolation of one coarse centre and one unknown.
// S(j, a, b): staged value (double).  Children: fine signed layer i in
// [-k, -1] at normal offset e_n = i + 2 (units of h), tangential offsets
// e0, e1 in {-1, 0, 1}.
// ---------------------------------------------------------------------------
template <int M, bool SPLIT, typename Stage, typename Out>
__device__ __forceinline__ void taylor_interp_task(const Stage& S, const Out& out, int k, int p, int a, int b) {
  using T = typename Arith<SPLIT>::T;
  const T* wt = Arith<SPLIT>::wt_interp();
  const int c[3] = {-1, a, b};
  const int lo[3] = {-k, 0, 0};
  const int hi[3] = {k - 1, p - 1, p - 1};
  int ps[3], pl[3], ms[3], ml[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    stencil_window(c[d], lo[d], hi[d], pure_exactness(M), ps[d], pl[d]);
    stencil_window(c[d], lo[d], hi[d], mixed_exactness(M), ms[d], ml[d]);
  }
  const double base = S(-1, a, b);
  // D(x): input value, or its difference to the base in SPLIT mode.
  auto D = [&](int j, int aa, int bb) -> T {
    const double v = S(j, aa, bb);
    if (SPLIT) return (T)(v - base);
    return (T)v;
  };
  auto W = [&](int L, int pos, int r) -> const T* { return wt + wt_offset(L) + (pos * 3 + r - 1) * L; };

  T C[M + 1][M + 1][M + 1];
#pragma unroll
  for (int x = 0; x <= M; ++x)
#pragma unroll
    for (int y = 0; y <= M; ++y)
#pragma unroll
      for (int z = 0; z <= M; ++z) C[x][y][z] = T(0);
  C[0][0][0] = SPLIT ? T(0) : (T)base;

  // pure derivatives along each axis
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int r = 1; r <= M; ++r) {
      const T* w = W(pl[d], c[d] - ps[d], r);
      T acc = T(0);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        if (i < pl[d]) {
          int x[3] = {c[0], c[1], c[2]};
          x[d] = ps[d] + i;
          acc += w[i] * D(x[0], x[1], x[2]);
        }
      }
      if (d == 0) C[r][0][0] = acc;
      if (d == 1) C[0][r][0] = acc;
      if (d == 2) C[0][0][r] = acc;
    }
  }
  // mixed derivatives over planes (d, e), orders (rd, re) with rd + re <= M
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int e = d + 1; e < 3; ++e)
#pragma unroll
      for (int rd = 1; rd < M; ++rd)
#pragma unroll
        for (int re = 1; re + rd <= M; ++re) {
          const T* wd = W(ml[d], c[d] - ms[d], rd);
          const T* we = W(ml[e], c[e] - ms[e], re);
          T acc = T(0);
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              int x[3] = {c[0], c[1], c[2]};
              x[d] = ms[d] + i;
              x[e] = ms[e] + q;
              acc += wd[i] * we[q] * D(x[0], x[1], x[2]);
            }
          int r3[3] = {0, 0, 0};
          r3[d] = rd;
          r3[e] = re;
          C[r3[0]][r3[1]][r3[2]] = acc;
        }
  if (M == 3) {  // u_{n t0 t1}
    const T* w0 = W(ml[0], c[0] - ms[0], 1);
    const T* w1 = W(ml[1], c[1] - ms[1], 1);
    const T* w2 = W(ml[2], c[2] - ms[2], 1);
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int q = 0; q < 3; ++q)
          acc += w0[i] * w1[j] * w2[q] * D(ms[0] + i, ms[1] + j, ms[2] + q);
    C[1][1][1] = acc;
  }

  // Evaluate at the children with even/odd splitting, axis by axis.
  // Step A (normal): R[y][z] at e_n in {-1, 0, +1}.
  Tri<T> R[M + 1][M + 1];
#pragma unroll
  for (int y = 0; y <= M; ++y)
#pragma unroll
    for (int z = 0; y + z <= M; ++z) {
      T ev = T(0), od = T(0);
#pragma unroll
      for (int x = 2; x + y + z <= M; x += 2) ev += C[x][y][z];
#pragma unroll
      for (int x = 1; x + y + z <= M; x += 2) od += C[x][y][z];
      const T c0 = C[0][y][z];
      R[y][z].z = c0;
      R[y][z].p = (c0 + ev) + od;
      R[y][z].m = (c0 + ev) - od;
    }
  // Children normal offsets: i = -1 -> +1, i = -2 -> 0, i = -3 -> -1.
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) {
    if (ii >= k) break;
    const int i = -1 - ii;
    // Step B (t0) for this e_n
    Tri<T> Sg[M + 1];
#pragma unroll
    for (int z = 0; z <= M; ++z) {
      auto pick = [&](const Tri<T>& t) -> T { return ii == 0 ? t.p : (ii == 1 ? t.z : t.m); };
      T ev = T(0), od = T(0);
#pragma unroll
      for (int y = 2; y + z <= M; y += 2) ev += pick(R[y][z]);
#pragma unroll
      for (int y = 1; y + z <= M; y += 2) od += pick(R[y][z]);
      const T c0 = pick(R[0][z]);
      Sg[z].z = c0;
      Sg[z].p = (c0 + ev) + od;
      Sg[z].m = (c0 + ev) - od;
    }
#pragma unroll
    for (int e0 = -1; e0 <= 1; ++e0) {
      T q[M + 1];
#pragma unroll
      for (int z = 0; z <= M; ++z) q[z] = e0 < 0 ? Sg[z].m : (e0 == 0 ? Sg[z].z : Sg[z].p);
      T ev = T(0), od = T(0);
#pragma unroll
      for (int z = 2; z <= M; z += 2) ev += q[z];
#pragma unroll
      for (int z = 1; z <= M; z += 2) od += q[z];
      const T vz = q[0], vp = (q[0] + ev) + od, vm = (q[0] + ev) - od;
      if (SPLIT) {
        out(i, a, b, e0, -1, base + (double)vm);
        out(i, a, b, e0, 0, (ii == 1 && e0 == 0) ? base : base + (double)vz);
        out(i, a, b, e0, 1, base + (double)vp);
      } else {
        out(i, a, b, e0, -1, (double)vm);
        out(i, a, b, e0, 0, (double)vz);
        out(i, a, b, e0, 1, (double)vp);
      }
    }
  }
}

// 1-D d-linear child values at offsets -1, 0, +1 from neighbours xm, x0, xp
// (coarse a-1, a, a+1); lo_edge / hi_edge: a has no neighbour below / above,
// so the missing bracket is replaced by linear extrapolation.
template <typename T>
__device__ __forceinline__ Tri<T> dlin3(T xm, T x0, T xp, bool lo_edge, bool hi_edge) {
  const T third = T(1) / T(3);
  Tri<T> r;
  r.z = x0;
  r.m = lo_edge ? (x0 + third * (x0 - xp)) : (x0 + third * (xm - x0));
  r.p = hi_edge ? (x0 + third * (x0 - xm)) : (x0 + third * (xp - x0));
  return r;
}

template <bool SPLIT, typename Stage, typename Out>
__device__ __forceinline__ void dlinear_interp_task(const Stage& S, const Out& out, int k, int p, int a, int b) {
  using T = typename Arith<SPLIT>::T;
  const double base = S(-1, a, b);
  auto D = [&](int j, int aa, int bb) -> T {
    const double v = S(j, aa, bb);
    if (SPLIT) return (T)(v - base);
    return (T)v;
  };
  const bool alo = a == 0, ahi = a == p - 1, blo = b == 0, bhi = b == p - 1;
  const int am = alo ? a : a - 1, ap = ahi ? a : a + 1;
  const int bm = blo ? b : b - 1, bp = bhi ? b : b + 1;
  const T third = T(1) / T(3);
  const int aidx[3] = {am, a, ap};
  const int bidx[3] = {bm, b, bp};
  // normal pass per tangential neighbour column: child layer -1 (offset +1/3 H
  // towards layer 0), -2 (coincident with layer -1), -3 (towards layer -2)
  T N[3][3][3];  // [child normal ii][da][db]
#pragma unroll
  for (int da = 0; da < 3; ++da)
#pragma unroll
    for (int db = 0; db < 3; ++db) {
      const T v1 = D(-1, aidx[da], bidx[db]);
      const T v0 = D(0, aidx[da], bidx[db]);
      N[0][da][db] = v1 + third * (v0 - v1);
      N[1][da][db] = v1;
      if (k >= 3) {
        const T v2 = D(-2, aidx[da], bidx[db]);
        N[2][da][db] = v1 + third * (v2 - v1);
      } else {
        N[2][da][db] = v1;
      }
    }
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) {
    if (ii >= k) break;
    const int i = -1 - ii;
    Tri<T> A[3];  // per db: children along t0
#pragma unroll
    for (int db = 0; db < 3; ++db) A[db] = dlin3<T>(N[ii][0][db], N[ii][1][db], N[ii][2][db], alo, ahi);
#pragma unroll
    for (int e0 = -1; e0 <= 1; ++e0) {
      auto pick = [&](const Tri<T>& t) -> T { return e0 < 0 ? t.m : (e0 == 0 ? t.z : t.p); };
      const Tri<T> r = dlin3<T>(pick(A[0]), pick(A[1]), pick(A[2]), blo, bhi);
      if (SPLIT) {
        out(i, a, b, e0, -1, base + (double)r.m);
        out(i, a, b, e0, 0, (ii == 1 && e0 == 0) ? base : base + (double)r.z);
        out(i, a, b, e0, 1, base + (double)r.p);
      } else {
        out(i, a, b, e0, -1, (double)r.m);
        out(i, a, b, e0, 0, (double)r.z);
        out(i, a, b, e0, 1, (double)r.p);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Interpolation kernel: one CTA per tile.
// ---------------------------------------------------------------------------
template <bool SPLIT>
__global__ void __launch_bounds__(256) interp_kernel(const amr_transfer_item* __restrict__ items,
                                                     const Tile* __restrict__ tiles, int U,
                                                     const double* __restrict__ coarse,
                                                     double* __restrict__ fine) {
  extern __shared__ double smem[];
  const Tile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  IRange rn, ra, rb;
  interp_region(p, k, m, t.a0, t.na, t.b0, t.nb, rn, ra, rb);
  const int NA = ra.hi - ra.lo + 1, NB = rb.hi - rb.lo + 1, NJ = rn.hi - rn.lo + 1;
  const int nu = t.nu;
  const int total = NJ * NB * NA * nu;
  const double* cb = coarse + it.coarse_offset + t.u0;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int u = e % nu;
    int v = e / nu;
    const int aa = v % NA;
    v /= NA;
    const int bb = v % NB;
    const int jj = v / NB;
    smem[e] = __ldg(cb + frame_vol(fr, rn.lo + jj, ra.lo + aa, rb.lo + bb) * U + u);
  }
  __syncthreads();
  const int64_t arr = fr.vols * U;
  double* fb = fine + it.fine_offset + (int64_t)t.slot * arr + t.u0;
  const int s0 = t.sub % 3, s1 = t.sub / 3;
  const int ntask = t.na * t.nb * nu;
  for (int e = threadIdx.x; e < ntask; e += blockDim.x) {
    const int u = e % nu;
    const int ci = e / nu;
    const int a = t.a0 + ci % t.na, b = t.b0 + ci / t.na;
    auto S = [&](int j, int aa, int bb) -> double {
      return smem[(((j - rn.lo) * NB + (bb - rb.lo)) * NA + (aa - ra.lo)) * nu + u];
    };
    auto O = [&](int i, int a_, int b_, int e0, int e1, double val) {
      const int q0 = 3 * a_ + 1 + e0 - s0 * p, q1 = 3 * b_ + 1 + e1 - s1 * p;
      fb[frame_vol(fr, i, q0, q1) * U + u] = val;
    };
    if (m == 3) taylor_interp_task<3, SPLIT>(S, O, k, p, a, b);
    else if (m == 2) taylor_interp_task<2, SPLIT>(S, O, k, p, a, b);
    else dlinear_interp_task<SPLIT>(S, O, k, p, a, b);
  }
}

// ---------------------------------------------------------------------------
// Restriction tasks: one coarse halo column (a, b), one unknown.  F(i, da, db)
// reads the fine volume at signed layer i, tangential offset (da, db) from the
// column coincident with the coarse centre; C(j, v) writes coarse halo layer j.
// ---------------------------------------------------------------------------
template <int M, bool SPLIT, typename Fine, typename Coarse>
__device__ __forceinline__ void taylor_restrict_task(const Fine& F, const Coarse& C, int k) {
  using T = typename Arith<SPLIT>::T;
  // k >= 2 (checked on the host): coarse layer 0 coincides with fine layer 1
  C(0, F(1, 0, 0));
  if (k < 2) return;
  int s, L;
  stencil_window(k - 1, -k, k - 1, pure_exactness(M), s, L);
  const double base = F(k - 1, 0, 0);
  const T* wt = Arith<SPLIT>::wt_restrict();
  const int pos = k - 1 - s;
  T cf[M + 1];
#pragma unroll
  for (int r = 1; r <= M; ++r) cf[r] = T(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i < L) {
      const double v = F(s + i, 0, 0);
      const T dv = SPLIT ? (T)(v - base) : (T)v;
#pragma unroll
      for (int r = 1; r <= M; ++r) cf[r] += wt[wt_offset(L) + (pos * 3 + r - 1) * L + i] * dv;
    }
  }
  for (int j = 1; j < k; ++j) {
    const T e = T(3 * j + 2 - k);  // offset from fine layer k-1 to coarse layer j, units of h
    T incr = cf[M];
#pragma unroll
    for (int r = M - 1; r >= 1; --r) incr = incr * e + cf[r];
    incr *= e;
    C(j, base + (double)incr);
  }
}

template <typename Fine, typename Coarse>
__device__ __forceinline__ void dlinear_restrict_task(const Fine& F, const Coarse& C, int k) {
  const int nl = k == 1 ? 2 : k;
  double avg[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (sl < nl) {
      const int i = k == 1 ? sl - 1 : sl;
      double acc = 0.0;
#pragma unroll
      for (int db = -1; db <= 1; ++db)
#pragma unroll
        for (int da = -1; da <= 1; ++da) acc += F(i, da, db);
      avg[sl] = acc * (1.0 / 9.0);
    }
  }
  for (int j = 0; j < k; ++j) {
    double v = 0.0;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl)
      if (sl < nl) v += c_ls[ls_index(k, j, sl)] * avg[sl];
    C(j, v);
  }
}

template <bool SPLIT>
__global__ void __launch_bounds__(256) restrict_kernel(const amr_transfer_item* __restrict__ items,
                                                       const Tile* __restrict__ tiles, int U,
                                                       const double* __restrict__ fine,
                                                       double* __restrict__ coarse) {
  const Tile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  const int64_t arr = fr.vols * U;
  const double* fb = fine + it.fine_offset + (int64_t)t.slot * arr + t.u0;
  double* cb = coarse + it.coarse_offset + t.u0;
  const int s0 = t.sub % 3, s1 = t.sub / 3;
  const int nu = t.nu;
  const int ntask = t.na * t.nb * nu;
  for (int e = threadIdx.x; e < ntask; e += blockDim.x) {
    const int u = e % nu;
    const int ci = e / nu;
    const int a = t.a0 + ci % t.na, b = t.b0 + ci / t.na;
    const int q0 = 3 * a + 1 - s0 * p, q1 = 3 * b + 1 - s1 * p;
    auto F = [&](int i, int da, int db) -> double {
      return __ldg(fb + frame_vol(fr, i, q0 + da, q1 + db) * U + u);
    };
    auto C = [&](int j, double v) { cb[frame_vol(fr, j, a, b) * U + u] = v; };
    // Restriction extrapolates up to (3k-1-(k-1))h = 5h away (k = 3), which
    // multiplies float32 rounding by up to ~125 (Taylor-3): it stays float64
    // in both precision modes.
    (void)SPLIT;
    if (m == 3) taylor_restrict_task<3, false>(F, C, k);
    else if (m == 2) taylor_restrict_task<2, false>(F, C, k);
    else dlinear_restrict_task(F, C, k);
  }
}

}  // namespace amr
