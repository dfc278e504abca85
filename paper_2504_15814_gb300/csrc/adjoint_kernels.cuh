// sm_103a kernels of the adjoint operators P^T and R^T (float64).
//
// P and R are linear (Q^f = P Q^c, Q^c = R Q^f, paper Sec. 2), so their
// adjoints are the transposed sparse operators.  The host assembles them per
// face class in the reference frame (orientation independent); the kernels
// gather: one thread per (output volume, unknown) sums its transposed row.
// No atomics: items that share a coarse face array are summed in item order,
// so results are deterministic.
#pragma once
#include "amr_common.cuh"
#include "builder.hpp"

namespace amr {

__device__ __forceinline__ int64_t packed_frame_vol(const FaceFrame& fr, uint32_t v, int k, int& slot) {
  slot = (int)(v >> 15);
  const int lk = (int)((v >> 12) & 7u), q1 = (int)((v >> 6) & 63u), q0 = (int)(v & 63u);
  return frame_vol(fr, lk - k, q0, q1);
}

// g_coarse = P^T g_fine for one group of items sharing a coarse face array.
__global__ void __launch_bounds__(256) interp_adjoint_kernel(
    const amr_transfer_item* __restrict__ items, const AdjointTile* __restrict__ tiles,
    const int32_t* __restrict__ group_ptr, const int32_t* __restrict__ group_items,
    const int32_t* __restrict__ item_class, const int32_t* __restrict__ cls_rows,
    const int32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col, const double* __restrict__ val,
    int U, const double* __restrict__ g_fine, double* __restrict__ g_coarse) {
  const AdjointTile t = tiles[blockIdx.x];
  const int m0 = group_ptr[t.index], m1 = group_ptr[t.index + 1];
  const amr_transfer_item first = items[group_items[m0]];
  const int p = first.patch_size, k = first.overlap;
  const FaceFrame fr = face_frame(first.face, p, k);
  const int64_t arrU = fr.vols * U;
  const int nu = t.nu;
  const int ntask = nu * p * p * 2 * k;
  for (int e = threadIdx.x; e < ntask; e += blockDim.x) {
    const int u = e % nu;
    const int r = e / nu;  // reference volume (lk p + q1) p + q0 of the coarse array
    const int q0 = r % p, q1 = (r / p) % p, lk = r / (p * p);
    double acc = 0.0;
    for (int mi = m0; mi < m1; ++mi) {
      const int item = group_items[mi];
      const double* gf = g_fine + items[item].fine_offset + t.u0 + u;
      const int32_t* rp = row_ptr + cls_rows[item_class[item]];
      for (int q = rp[r]; q < rp[r + 1]; ++q) {
        int slot;
        const int64_t vol = packed_frame_vol(fr, col[q], k, slot);
        acc = fma(val[q], __ldg(gf + slot * arrU + vol * U), acc);
      }
    }
    g_coarse[first.coarse_offset + frame_vol(fr, lk - k, q0, q1) * U + t.u0 + u] = acc;
  }
}

// g_fine = R^T g_coarse for one fine face array of one item.
__global__ void __launch_bounds__(256) restrict_adjoint_kernel(
    const amr_transfer_item* __restrict__ items, const AdjointTile* __restrict__ tiles,
    const int32_t* __restrict__ cls_rows, const int32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const double* __restrict__ val, int U, const double* __restrict__ g_coarse, double* __restrict__ g_fine) {
  const AdjointTile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.index];
  const int p = it.patch_size, k = it.overlap;
  const FaceFrame fr = face_frame(it.face, p, k);
  const int64_t arrU = fr.vols * U;
  const int nvol = p * p * 2 * k;
  const int32_t* rp = row_ptr + cls_rows[t.klass] + t.slot * nvol;
  const double* gc = g_coarse + it.coarse_offset + t.u0;
  double* gf = g_fine + it.fine_offset + t.slot * arrU + t.u0;
  const int nu = t.nu;
  const int ntask = nu * nvol;
  for (int e = threadIdx.x; e < ntask; e += blockDim.x) {
    const int u = e % nu;
    const int r = e / nu;
    const int q0 = r % p, q1 = (r / p) % p, lk = r / (p * p);
    double acc = 0.0;
    for (int q = rp[r]; q < rp[r + 1]; ++q) {
      int slot;
      const int64_t vol = packed_frame_vol(fr, col[q], k, slot);
      acc = fma(val[q], __ldg(gc + vol * U + u), acc);
    }
    gf[frame_vol(fr, lk - k, q0, q1) * U + u] = acc;
  }
}

}  // namespace amr
