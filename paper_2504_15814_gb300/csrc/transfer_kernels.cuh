// sm_103a kernels of the coarse<->fine transfer (forward operators).
//
// Work decomposition: one CTA per tile (a rectangle of coarse columns of one
// subface, and a range of unknowns).  Interpolation stages the tile's stencil
// region of the coarse face array in shared memory with coalesced loads along
// the AoS unknown axis, then one thread per (coarse centre, unknown) computes
// the centre's Taylor coefficients (or d-linear partial sums) and writes its
// k * 3 * 3 fine children.  The restriction kernel (restrict_kernels.cuh)
// needs no staging: one thread per (coarse halo column, unknown) reads the
// coincident fine normal line.
//
// Precision: FP64 computes everything in float64.  SPLIT keeps float64
// instructions out of the kernels: inputs are split exactly into float pairs,
// differences to the base value are formed from the pairs, interpolation
// increments are float32, Taylor restriction (large extrapolation weights)
// uses float-pair arithmetic, and outputs are rebuilt as float64 by integer
// assembly.
#pragma once
#include "amr_common.cuh"
#include "split_arith.cuh"
#include "builder.hpp"

#include <type_traits>

namespace amr {

// Largest CTA of the split-precision interpolation kernel (two CTAs per SM
// keep about 80 registers per thread).
constexpr int kMaxSplitInterpThreads = 384;

__constant__ double c_wt_interp[WT_SIZE];
__constant__ double c_wt_restrict[WT_SIZE];
__constant__ float c_wt_interp_f[WT_SIZE];
__constant__ float c_wt_restrict_f[WT_SIZE];
__constant__ double c_ls[LS_SIZE];
__constant__ float c_ls_f[LS_SIZE];
__constant__ double c_rw[RW_SIZE];
__constant__ float c_rw_hi[RW_SIZE];
__constant__ float c_rw_lo[RW_SIZE];

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

// Evaluate the Taylor polynomial with coefficients C (units of the fine
// spacing) at the children of a coarse centre, by even/odd splitting, axis by
// axis; emit(ii, e0, e1, v) as for taylor_interp_core.
template <int M, typename T, typename Emit>
__device__ __forceinline__ void taylor_children(const T (&C)[M + 1][M + 1][M + 1], const Emit& emit, int k) {
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
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) {
    if (ii >= k) break;
    auto pick = [&](const Tri<T>& t) -> T { return ii == 0 ? t.p : (ii == 1 ? t.z : t.m); };
    Tri<T> Sg[M + 1];  // Step B (t0) for this normal offset
#pragma unroll
    for (int z = 0; z <= M; ++z) {
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
    for (int e0 = -1; e0 <= 1; ++e0) {  // Step C (t1)
      T q[M + 1];
#pragma unroll
      for (int z = 0; z <= M; ++z) q[z] = e0 < 0 ? Sg[z].m : (e0 == 0 ? Sg[z].z : Sg[z].p);
      T ev = T(0), od = T(0);
#pragma unroll
      for (int z = 2; z <= M; z += 2) ev += q[z];
#pragma unroll
      for (int z = 1; z <= M; z += 2) od += q[z];
      emit(ii, e0, -1, (q[0] + ev) - od);
      emit(ii, e0, 0, q[0]);
      emit(ii, e0, 1, (q[0] + ev) + od);
    }
  }
}


// ---------------------------------------------------------------------------
// Taylor-m interpolation of one coarse centre (layer cl, a, b) and one
// unknown.  D(j, a', b') returns the input value (float64 path) or its
// difference to the centre value (split path); c000 is the centre value or 0.
// emit(ii, e0, e1, v) receives the Taylor value (or increment) of the child
// ii < kk below the centre (normal offset +1, 0, -1 for ii = 0, 1, 2, units
// of h; fine signed layer -1-ii for cl = -1) and tangential offsets e0, e1 in
// {-1, 0, 1}.
// ---------------------------------------------------------------------------
template <int M, typename T, typename Diff>
__device__ __forceinline__ void taylor_interp_coeffs(const Diff& D, const T* __restrict__ wt, int k, int p, int a,
                                                     int b, T c000, int cl, T (&C)[M + 1][M + 1][M + 1]) {
  const int c[3] = {cl, a, b};
  const int lo[3] = {-k, 0, 0};
  const int hi[3] = {k - 1, p - 1, p - 1};
  int ps[3], pl[3], ms[3], ml[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    stencil_window(c[d], lo[d], hi[d], pure_exactness(M), ps[d], pl[d]);
    stencil_window(c[d], lo[d], hi[d], mixed_exactness(M), ms[d], ml[d]);
  }
  auto W = [&](int L, int pos, int r) -> const T* { return wt + wt_offset(L) + (pos * 3 + r - 1) * L; };

#pragma unroll
  for (int x = 0; x <= M; ++x)
#pragma unroll
    for (int y = 0; y <= M; ++y)
#pragma unroll
      for (int z = 0; z <= M; ++z) C[x][y][z] = T(0);
  C[0][0][0] = c000;

  // pure derivatives along each axis: one pass over the window, all orders
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* w1 = W(pl[d], c[d] - ps[d], 1);
    T acc[M + 1];
#pragma unroll
    for (int r = 1; r <= M; ++r) acc[r] = T(0);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (i < pl[d]) {
        int x[3] = {c[0], c[1], c[2]};
        x[d] = ps[d] + i;
        const T v = D(x[0], x[1], x[2]);
#pragma unroll
        for (int r = 1; r <= M; ++r) acc[r] += w1[(r - 1) * pl[d] + i] * v;
      }
    }
#pragma unroll
    for (int r = 1; r <= M; ++r) {
      if (d == 0) C[r][0][0] = acc[r];
      if (d == 1) C[0][r][0] = acc[r];
      if (d == 2) C[0][0][r] = acc[r];
    }
  }
  // Mixed derivatives.  Every axis's mixed window has 3 points (ms[d] ..
  // ms[d] + 2) for Taylor orders, so all of them come from one 3x3x3 box of
  // values, collapsed axis by axis: along the normal into (value at c, r = 1,
  // r = 2) -- the normal window is centred on the centre's layer, as
  // 2k >= m + 1 >= 3 and a second centre layer exists only for k >= 4 --
  // then along t0 into (value at c, r = 1, r = 2) with c's box index sa, then
  // along t1 likewise.  Each box value is read once.
  {
    const T* wn = W(3, c[0] - ms[0], 1);  // rows r = 1, 2 at +0, +3
    const T* wa = W(3, c[1] - ms[1], 1);
    const T* wb = W(3, c[2] - ms[2], 1);
    const int sa = c[1] - ms[1], sb = c[2] - ms[2];
    T m110 = T(0), m011 = T(0), m101 = T(0);                          // second order
    T m210 = T(0), m120 = T(0), m201 = T(0), m102 = T(0), m021 = T(0), m012 = T(0), m111 = T(0);  // third
#pragma unroll
    for (int q = 0; q < 3; ++q) {  // t1 index in the box
      T p11 = T(0), p10 = T(0), p01 = T(0), p21 = T(0), p12 = T(0), p20 = T(0), p02 = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {  // t0 index in the box
        const T x0 = D(ms[0], ms[1] + j, ms[2] + q);
        const T x1 = D(ms[0] + 1, ms[1] + j, ms[2] + q);
        const T x2 = D(ms[0] + 2, ms[1] + j, ms[2] + q);
        const T s1 = wn[0] * x0 + wn[1] * x1 + wn[2] * x2;  // d/dn
        const T a1 = wa[j];
        p11 += a1 * s1;
        p01 += a1 * x1;  // x1: the normal point at c
        if (j == sa) p10 = s1;  // point evaluation at c along t0: a select, no arithmetic
        if (M == 3) {
          const T s2 = wn[3] * x0 + wn[4] * x1 + wn[5] * x2;  // d2/dn2
          const T a2 = wa[3 + j];
          p21 += a1 * s2;
          p12 += a2 * s1;
          p02 += a2 * x1;
          if (j == sa) p20 = s2;
        }
      }
      const T b1 = wb[q];
      if (q == sb) m110 = p11;  // point evaluation at c along t1
      m101 += b1 * p10;
      m011 += b1 * p01;
      if (M == 3) {
        const T b2 = wb[3 + q];
        if (q == sb) {
          m210 = p21;
          m120 = p12;
        }
        m201 += b1 * p20;
        m102 += b2 * p10;
        m021 += b1 * p02;
        m012 += b2 * p01;
        m111 += b1 * p11;
      }
    }
    C[1][1][0] = m110;
    C[1][0][1] = m101;
    C[0][1][1] = m011;
    if (M == 3) {
      C[2][1][0] = m210;
      C[1][2][0] = m120;
      C[2][0][1] = m201;
      C[1][0][2] = m102;
      C[0][2][1] = m021;
      C[0][1][2] = m012;
      C[1][1][1] = m111;
    }
  }

}

// Taylor coefficients (units of the fine spacing, the centre value c000
// included) of the coarse centre (cl, a, b), evaluated at its children.
template <int M, typename T, typename Diff, typename Emit>
__device__ __forceinline__ void taylor_interp_core(const Diff& D, const Emit& emit, const T* __restrict__ wt,
                                                   int k, int p, int a, int b, T c000, int cl = -1,
                                                   int kk = 3) {
  T C[M + 1][M + 1][M + 1];
  taylor_interp_coeffs<M, T>(D, wt, k, p, a, b, c000, cl, C);
  taylor_children<M, T>(C, emit, kk < k ? kk : k);
}

// Least-squares Taylor-m interpolation of one coarse centre (scheme 1; the
// paper's fit of all derivatives at once, Sec. 3): the derivatives are
// W^T d over the slots of the finite-difference stencils (the pure lines and
// the 3x3x3 box of the mixed windows, slot layout in amr_common.cuh), W the
// host's fit for the centre's class.  D, emit and c000 as for
// taylor_interp_core; with RAW (float64 path) D returns input values rather
// than differences, so c000 times the column sums of W is subtracted.
template <int M, bool RAW, typename T, typename Diff, typename Emit>
__device__ __forceinline__ void ls_interp_core(const Diff& D, const Emit& emit, const T* __restrict__ wcls,
                                               const T* __restrict__ wsum, int k, int p, int a, int b, T c000) {
  constexpr int NA = M == 3 ? 19 : 9;
  const int c[3] = {-1, a, b};
  const int lo[3] = {-k, 0, 0};
  const int hi[3] = {k - 1, p - 1, p - 1};
  int ps[3], pl[3], ms[3], ml[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    stencil_window(c[d], lo[d], hi[d], pure_exactness(M), ps[d], pl[d]);
    stencil_window(c[d], lo[d], hi[d], mixed_exactness(M), ms[d], ml[d]);
  }
  T acc[NA];
#pragma unroll
  for (int al = 0; al < NA; ++al) acc[al] = T(0);
  auto add = [&](int slot, T v) {
#pragma unroll
    for (int al = 0; al < NA; ++al) acc[al] += __ldg(wcls + slot * LS_NALPHA + al) * v;
  };
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (i < pl[d]) {
        int x[3] = {c[0], c[1], c[2]};
        x[d] = ps[d] + i;
        add(d * 5 + i, D(x[0], x[1], x[2]));
      }
  const int sa = c[1] - ms[1], sb = c[2] - ms[2];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        // Taylor-2 uses only the three planes through the centre (the normal
        // window is centred on layer -1: i == 1)
        if (M == 3 || i == 1 || j == sa || q == sb) add(15 + (q * 3 + j) * 3 + i, D(ms[0] + i, ms[1] + j, ms[2] + q));
  if (RAW) {
#pragma unroll
    for (int al = 0; al < NA; ++al) acc[al] -= __ldg(wsum + al) * c000;
  }
  T C[M + 1][M + 1][M + 1];
#pragma unroll
  for (int x = 0; x <= M; ++x)
#pragma unroll
    for (int y = 0; y <= M; ++y)
#pragma unroll
      for (int z = 0; z <= M; ++z) C[x][y][z] = T(0);
  C[0][0][0] = c000;
  int al = 0;  // the host's derivative order: x, then y, then z ascending
#pragma unroll
  for (int x = 0; x <= M; ++x)
#pragma unroll
    for (int y = 0; x + y <= M; ++y)
#pragma unroll
      for (int z = 0; x + y + z <= M; ++z)
        if (x + y + z > 0) C[x][y][z] = acc[al++];
  taylor_children<M, T>(C, emit, k);
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

// d-linear interpolation of one coarse centre: the normal lerp on the 3x3
// neighbour columns, then along t0, then along t1 (the tensor product
// P = P_t1 P_t0 P_n of Sec. 2, sum-factorised).  Same D / emit contract.
template <typename T, typename Diff, typename Emit>
__device__ __forceinline__ void dlinear_interp_core(const Diff& D, const Emit& emit, int k, int p, int a, int b,
                                                    int cl = -1, int kk = 3) {
  if (kk > k) kk = k;
  const bool alo = a == 0, ahi = a == p - 1, blo = b == 0, bhi = b == p - 1;
  const int aidx[3] = {alo ? a : a - 1, a, ahi ? a : a + 1};
  const int bidx[3] = {blo ? b : b - 1, b, bhi ? b : b + 1};
  const T third = T(1) / T(3);
  T N[3][3][3];  // [child normal ii][da][db]
#pragma unroll
  for (int da = 0; da < 3; ++da)
#pragma unroll
    for (int db = 0; db < 3; ++db) {
      const T v1 = D(cl, aidx[da], bidx[db]);
      const T v0 = D(cl + 1, aidx[da], bidx[db]);
      N[0][da][db] = v1 + third * (v0 - v1);  // child above the centre: towards coarse layer cl + 1
      N[1][da][db] = v1;                      // child coincident with coarse layer cl
      N[2][da][db] = v1;
      if (kk >= 3) N[2][da][db] = v1 + third * (D(cl - 1, aidx[da], bidx[db]) - v1);  // child below
    }
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) {
    if (ii >= kk) break;
    Tri<T> A[3];
#pragma unroll
    for (int db = 0; db < 3; ++db) A[db] = dlin3<T>(N[ii][0][db], N[ii][1][db], N[ii][2][db], alo, ahi);
#pragma unroll
    for (int e0 = -1; e0 <= 1; ++e0) {
      auto pick = [&](const Tri<T>& t) -> T { return e0 < 0 ? t.m : (e0 == 0 ? t.z : t.p); };
      const Tri<T> r = dlin3<T>(pick(A[0]), pick(A[1]), pick(A[2]), blo, bhi);
      emit(ii, e0, -1, r.m);
      emit(ii, e0, 0, r.z);
      emit(ii, e0, 1, r.p);
    }
  }
}

// Where the fine children of coarse centre (a, b) live: the fine face array
// (slot) and the offset of tangential index 0 of that subface.
struct ChildMap {
  int slot, q0_off, q1_off;
};
__device__ __forceinline__ ChildMap child_map(const Tile& t, int p, int a, int b) {
  ChildMap m;
  int s0, s1;
  if (t.sub >= 0) {
    s0 = t.sub % 3;
    s1 = t.sub / 3;
    m.slot = t.slot;
  } else {  // whole-face tile: the subface follows from the centre;
            // (a + 1/2) / w is never within 1/32 of an integer (w <= 16)
    const float inv_w = 3.0f / (float)p;
    s0 = (int)(((float)a + 0.5f) * inv_w);
    s1 = (int)(((float)b + 0.5f) * inv_w);
    m.slot = s0 + 3 * s1;
  }
  m.q0_off = 1 - s0 * p;
  m.q1_off = 1 - s1 * p;
  return m;
}

// Patch sizes that are not a multiple of 3: placement of the children
// e = -1, 0, +1 of a coarse centre along one tangential axis, relative to the
// centre child (fine global g = 3a + 1, local q in the subface array it is
// addressed in).  In a whole-face tile the centre child's own array is used
// and an outer child on the far side of a subface boundary steps into the
// neighbouring array (slot_stride apart, local index p - 1 or 0).  In a
// one-subface tile every child outside [0, p) is dropped.
struct CutAxis {
  long long off_m, off_p;
  bool v_m, v_z, v_p;
};
__device__ __forceinline__ CutAxis cut_axis(bool whole, int q, int p, long long gs, long long slot_stride) {
  CutAxis c;
  c.off_m = (whole && q == 0) ? (long long)(p - 1) * gs - slot_stride : -gs;
  c.off_p = (whole && q == p - 1) ? slot_stride - (long long)(p - 1) * gs : gs;
  c.v_m = whole || (q >= 1 && q <= p);
  c.v_z = whole || (q >= 0 && q < p);
  c.v_p = whole || (q >= -1 && q <= p - 2);
  return c;
}
__device__ __forceinline__ long long cut_off(const CutAxis& c, int e) { return e < 0 ? c.off_m : (e > 0 ? c.off_p : 0); }
__device__ __forceinline__ bool cut_valid(const CutAxis& c, int e) { return e < 0 ? c.v_m : (e > 0 ? c.v_p : c.v_z); }

// Mixed-radix counter over (u, x, y, z) with radices (nu, NX, NY, -): walks
// e, e + step, ... without integer divisions in the loop.
struct Counter4 {
  int u, x, y, z;
  int su, sx, sy, sz;
  __device__ void init(int e, int step, int nu, int NX, int NY) {
    u = e % nu; int v = e / nu; x = v % NX; v /= NX; y = v % NY; z = v / NY;
    su = step % nu; int w = step / nu; sx = w % NX; w /= NX; sy = w % NY; sz = w / NY;
  }
  __device__ __forceinline__ void advance(int nu, int NX, int NY) {
    u += su; int c = u >= nu; u -= c ? nu : 0;
    x += sx + c; c = x >= NX; x -= c ? NX : 0;
    y += sy + c; c = y >= NY; y -= c ? NY : 0;
    z += sz + c;
  }
};

// ---------------------------------------------------------------------------
// Interpolation kernel: one CTA per tile (a rectangle of coarse centres of one
// face and a chunk of unknowns).  Phase 1 stages the stencil region in shared
// memory (float64, or exact float pairs in split mode); phase 2 runs one thread
// per (centre, unknown).
// Split mode: the stencil differences come from the pairs and the derivative
// and Taylor arithmetic is float32; the child coincident with the centre is
// the centre's own float64 value; the other children are rebuilt as float64
// from base + increment, either by one float64 add of the exactly converted
// increment or by TwoSum + integer assembly without any float64 instruction.
// The share of each (ADDBACK) balances the GB300 float64 unit (about 1/73 of
// the float32 rate) against the integer issue slots; the autotuner picks it.
// ---------------------------------------------------------------------------
// ADDBACK (split mode): which children add the increment with one float64
// add (the rest use the integer assembly): 0 none, 1 e0 <= 0 and e1 <= 0
// (4/9), 2 e1 <= 0 (2/3), 3 all but e0 = e1 = +1 (8/9).
// INCR (split mode): write the float32 increments (layout of
// amr_transfer_plan_interpolate_increments) instead of float64 fine values.
// CUT: tiles of items whose patch size is not a multiple of 3 (children of
// one centre may lie in two fine face arrays, see CutAxis).
// lanes: 0 packs the (centre, unknown) tasks densely, unknown fastest; 32
// gives each coarse centre one warp, lane = unknown (tiles carry <= 32
// unknowns), so the per-centre window and weight work is warp-uniform.
// LS: least-squares derivatives (scheme 1) from the tables ls_wf / ls_wd at
// the item's block ls_off[item].
template <bool SPLIT, int ADDBACK = 2, bool INCR = false, bool CUT = false, bool LS = false>
__global__ void __launch_bounds__(SPLIT ? kMaxSplitInterpThreads : 256, 2)
    interp_kernel(const amr_transfer_item* __restrict__ items, const Tile* __restrict__ tiles, int U,
                  const double* __restrict__ coarse, double* __restrict__ fine, float* __restrict__ incr,
                  const int64_t* __restrict__ incr_off, int lanes, const float* __restrict__ ls_wf = nullptr,
                  const double* __restrict__ ls_wd = nullptr, const int64_t* __restrict__ ls_off = nullptr) {
  using SType = typename std::conditional<SPLIT, F2, double>::type;
  extern __shared__ double smem_raw[];
  SType* sm = reinterpret_cast<SType*>(smem_raw);
  const Tile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int p = it.patch_size, k = it.overlap, m = it.order;
  const FaceFrame fr = face_frame(it.face, p, k);
  IRange rn, ra, rb;
  interp_region(p, k, m, t.a0, t.na, t.b0, t.nb, rn, ra, rb);
  const int NA = ra.hi - ra.lo + 1, NB = rb.hi - rb.lo + 1, NJ = rn.hi - rn.lo + 1;
  const int nu = t.nu;
  // 32-bit element strides inside one face array (< 2^31 elements, checked on the host)
  const int gs_n = (int)fr.s_n * U, gs_a = (int)fr.s_t0 * U, gs_b = (int)fr.s_t1 * U;
  const double* cb = coarse + it.coarse_offset + t.u0;
  {
    const double* g0 = cb + frame_vol(fr, rn.lo, ra.lo, rb.lo) * U;
    const int total = NJ * NB * NA * nu;
    Counter4 c;
    c.init(threadIdx.x, blockDim.x, nu, NA, NB);
    // batches of STAGE loads in flight per thread before any conversion
    constexpr int STAGE = 8;
    for (int e0 = threadIdx.x; e0 < total; e0 += STAGE * blockDim.x) {
      double v[STAGE];
#pragma unroll
      for (int q = 0; q < STAGE; ++q) {
        if (e0 + q * (int)blockDim.x < total) v[q] = __ldg(g0 + c.z * gs_n + c.y * gs_b + c.x * gs_a + c.u);
        c.advance(nu, NA, NB);
      }
#pragma unroll
      for (int q = 0; q < STAGE; ++q) {
        const int e = e0 + q * blockDim.x;
        if (e < total) {
          if constexpr (SPLIT) sm[e] = split_f64(v[q]);
          else sm[e] = v[q];
        }
      }
    }
  }
  __syncthreads();
  const int64_t arr = fr.vols * U;
  const float inv_p = 1.0f / (float)p;
  const int SA = nu, SB = NA * nu, SJ = NB * NA * nu;
  // task walk: (unknown, centre) pairs, or centres only with the lane as the unknown
  const bool per_warp = lanes == 32;
  const int lane = threadIdx.x & 31;
  const int w_nu = per_warp ? 1 : nu;
  const int e_first = per_warp ? (int)(threadIdx.x >> 5) : (int)threadIdx.x;
  const int e_step = per_warp ? (int)(blockDim.x >> 5) : (int)blockDim.x;
  const int ntask = t.na * t.nb * w_nu * centre_layers(k);  // centres (a, b) of each centre layer
  Counter4 c;
  c.init(e_first, e_step, w_nu, t.na, t.nb);
  for (int e = (per_warp && lane >= nu) ? ntask : e_first; e < ntask; e += e_step, c.advance(w_nu, t.na, t.nb)) {
    const int u = per_warp ? lane : c.u, a = t.a0 + c.x, b = t.b0 + c.y;
    const int cl = -1 - c.z, kk = child_layers(k, c.z);  // centre layer and its child layers
    ChildMap cm;
    CutAxis ca, cbx;
    if constexpr (CUT) {
      // the centre child's subface: 3a + 1 = s p + q, 0 <= q < p in a whole-face tile
      int s0 = t.sub % 3, s1 = t.sub / 3;
      cm.slot = t.slot;
      if (t.sub < 0) {
        s0 = (int)(__fmaf_rn((float)a, 3.f, 1.5f) * inv_p);
        s1 = (int)(__fmaf_rn((float)b, 3.f, 1.5f) * inv_p);
        cm.slot = s0 + 3 * s1;
      }
      cm.q0_off = 1 - s0 * p;
      cm.q1_off = 1 - s1 * p;
      // strides of the written layout: fine face arrays, or the increment array
      const long long g0s = INCR ? (long long)U : gs_a, g1s = INCR ? (long long)p * U : gs_b;
      const long long slot_s = INCR ? (long long)k * p * p * U : arr;
      ca = cut_axis(t.sub < 0, 3 * a + cm.q0_off, p, g0s, slot_s);
      cbx = cut_axis(t.sub < 0, 3 * b + cm.q1_off, p, g1s, 3 * slot_s);
    } else {
      cm = child_map(t, p, a, b);
    }
    // child ii = 0 (fine layer -1 - 3 c.z, tangential offsets 0, 0) of this centre and unknown
    double* fc = fine + it.fine_offset + (int64_t)cm.slot * arr +
                 frame_vol(fr, cl - 2 * c.z, 3 * a + cm.q0_off, 3 * b + cm.q1_off) * U + t.u0 + u;
    const int ic = ((cl - rn.lo) * NB + (b - rb.lo)) * NA * nu + (a - ra.lo) * nu + u;
    auto S = [&](int j, int aa, int bb) -> SType { return sm[ic + (j - cl) * SJ + (bb - b) * SB + (aa - a) * SA]; };
    auto store = [&](int ii, int e0, int e1, double v) {
      if constexpr (CUT) {
        if (cut_valid(ca, e0) && cut_valid(cbx, e1)) fc[-ii * gs_n + cut_off(ca, e0) + cut_off(cbx, e1)] = v;
      } else {
        fc[-ii * gs_n + e0 * gs_a + e1 * gs_b] = v;
      }
    };
    if constexpr (SPLIT) {
      const F2 hc = sm[ic];
      const double base = __ldg(cb + frame_vol(fr, cl, a, b) * U + u);
      auto D = [&](int j, int aa, int bb) -> float {
        const F2 x = S(j, aa, bb);
        return __fadd_rn(__fsub_rn(x.hi, hc.hi), __fsub_rn(x.lo, hc.lo));
      };
      // increment layout: item offset + (((slot k + g) p + q1) p + q0) U + u
      float* ic_out = nullptr;
      if constexpr (INCR)
        ic_out = incr + incr_off[t.item] +
                 ((((int64_t)cm.slot * k) * p + (3 * b + cm.q1_off)) * p + (3 * a + cm.q0_off)) * U + t.u0 + u;
      auto emit = [&](int ii, int e0, int e1, float incr_v) {
        if constexpr (INCR) {
          const float w = (ii == 1 && e0 == 0 && e1 == 0) ? 0.f : incr_v;
          if constexpr (CUT) {
            if (cut_valid(ca, e0) && cut_valid(cbx, e1)) ic_out[(long long)ii * p * p * U + cut_off(ca, e0) + cut_off(cbx, e1)] = w;
          } else {
            ic_out[((ii * p + e1) * p + e0) * U] = w;
          }
          return;
        }
        const float incr = incr_v;
        double v;
        if (ii == 1 && e0 == 0 && e1 == 0) v = base;
        else if ((ADDBACK == 1 && e0 <= 0 && e1 <= 0) || (ADDBACK == 2 && e1 <= 0) ||
                 (ADDBACK == 3 && (e0 < 1 || e1 < 1)))
          v = __dadd_rn(base, f32_to_f64(incr));
        else v = add_back(hc, incr);
        store(ii, e0, e1, v);
      };
      if constexpr (LS) {
        const int cls = ls_class(a, p) + 5 * ls_class(b, p);
        const float* wb = ls_wf + ls_off[t.item];
        const float* wc = wb + cls * LS_SLOTS * LS_NALPHA;
        const float* ws = wb + LS_CLASSES * LS_SLOTS * LS_NALPHA + cls * LS_NALPHA;
        if (m == 3) ls_interp_core<3, false, float>(D, emit, wc, ws, k, p, a, b, 0.f);
        else ls_interp_core<2, false, float>(D, emit, wc, ws, k, p, a, b, 0.f);
      } else {
        if (m == 3) taylor_interp_core<3, float>(D, emit, c_wt_interp_f, k, p, a, b, 0.f, cl, kk);
        else if (m == 2) taylor_interp_core<2, float>(D, emit, c_wt_interp_f, k, p, a, b, 0.f, cl, kk);
        else dlinear_interp_core<float>(D, emit, k, p, a, b, cl, kk);
      }
    } else {
      auto emit = [&](int ii, int e0, int e1, double v) { store(ii, e0, e1, v); };
      if constexpr (LS) {
        const int cls = ls_class(a, p) + 5 * ls_class(b, p);
        const double* wb = ls_wd + ls_off[t.item];
        const double* wc = wb + cls * LS_SLOTS * LS_NALPHA;
        const double* ws = wb + LS_CLASSES * LS_SLOTS * LS_NALPHA + cls * LS_NALPHA;
        if (m == 3) ls_interp_core<3, true, double>(S, emit, wc, ws, k, p, a, b, S(-1, a, b));
        else ls_interp_core<2, true, double>(S, emit, wc, ws, k, p, a, b, S(-1, a, b));
      } else {
        if (m == 3) taylor_interp_core<3, double>(S, emit, c_wt_interp, k, p, a, b, S(cl, a, b), cl, kk);
        else if (m == 2) taylor_interp_core<2, double>(S, emit, c_wt_interp, k, p, a, b, S(cl, a, b), cl, kk);
        else dlinear_interp_core<double>(S, emit, k, p, a, b, cl, kk);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// fine ghost value = nearest coarse centre value + float32 increment.  One
// thread per (ghost volume, unknown) of one fine face array; even warps add in
// float64 (exact conversion + DADD), odd warps by TwoSum + integer assembly,
// sharing the float64 unit and the integer pipes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) apply_increments_kernel(const amr_transfer_item* __restrict__ items,
                                                               const AdjointTile* __restrict__ tiles,
                                                               const int64_t* __restrict__ incr_off, int U,
                                                               const double* __restrict__ coarse,
                                                               const float* __restrict__ incr,
                                                               double* __restrict__ fine) {
  const AdjointTile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.index];
  const int p = it.patch_size, k = it.overlap;
  const FaceFrame fr = face_frame(it.face, p, k);
  const int64_t arr = fr.vols * U;
  const int sub = it.subface < 0 ? t.slot : it.subface;
  const int s0 = sub % 3, s1 = sub / 3;
  const float* ib = incr + incr_off[t.index] + (int64_t)t.slot * k * p * p * U + t.u0;
  double* fb = fine + it.fine_offset + (int64_t)t.slot * arr + t.u0;
  const double* cb = coarse + it.coarse_offset + t.u0;
  const int nu = t.nu;
  const int ntask = nu * p * p * k;
  const bool f64_warp = ((threadIdx.x >> 5) & 1) == 0;
  Counter4 c;
  c.init(threadIdx.x, blockDim.x, nu, p, p);
  for (int e = threadIdx.x; e < ntask; e += blockDim.x, c.advance(nu, p, p)) {
    const int u = c.u, q0 = c.x, q1 = c.y, g = c.z;
    const int a = (s0 * p + q0) / 3, b = (s1 * p + q1) / 3;
    const double base = __ldg(cb + frame_vol(fr, -1, a, b) * U + u);
    const float d = __ldg(ib + ((g * p + q1) * p + q0) * U + u);
    double v;
    if (d == 0.f) v = base;
    else if (f64_warp) v = __dadd_rn(base, f32_to_f64(d));
    else v = add_back(split_f64(base), d);
    fb[frame_vol(fr, -1 - g, q0, q1) * U + u] = v;
  }
}

}  // namespace amr
