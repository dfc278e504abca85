// sm_103a kernel applying explicit sparse operator rows (CSR, the paper's own
// storage, Sec. 4.2): used for the least-squares scheme and, with
// AMR_FLAG_CSR, for every item (a baseline of the paper's design on the GPU).
//
// One warp per row, lanes over the unknowns of the AoS layout (Sec. 4.2
// vectorises over the 58 unknowns the same way): the row's entries are
// uniform across the warp, the input loads of a lane group are contiguous.
#pragma once
#include "amr_common.cuh"
#include "builder.hpp"
#include "split_arith.cuh"

namespace amr {

__device__ __forceinline__ int64_t csr_vol(const FaceFrame& fr, uint32_t v, int k, int& slot) {
  slot = (int)(v >> 15);
  return frame_vol(fr, (int)((v >> 12) & 7u) - k, (int)(v & 63u), (int)((v >> 6) & 63u));
}

// INTERP: rows of P (coarse -> fine ghosts), else rows of R (fine -> coarse
// halo).  SPLIT applies to interpolation rows: float32 weights on exact float-
// pair differences to the row's base value, float64 rebuilt without float64
// instructions; restriction rows (extrapolation weights up to ~10^2) and the
// FP64 mode accumulate in float64.
template <bool SPLIT, bool INTERP>
__global__ void __launch_bounds__(256) csr_apply_kernel(const amr_transfer_item* __restrict__ items,
                                                        const CsrTile* __restrict__ tiles,
                                                        const int32_t* __restrict__ row_ptr,
                                                        const uint32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const float* __restrict__ val_f,
                                                        const uint32_t* __restrict__ out_vol,
                                                        const uint32_t* __restrict__ base_vol, int U,
                                                        const double* __restrict__ in, double* __restrict__ out) {
  const CsrTile t = tiles[blockIdx.x];
  const amr_transfer_item it = items[t.item];
  const int k = it.overlap;
  const FaceFrame fr = face_frame(it.face, it.patch_size, k);
  const int64_t arrU = fr.vols * U;
  const double* ib = in + (INTERP ? it.coarse_offset : it.fine_offset);
  double* ob = out + (INTERP ? it.fine_offset : it.coarse_offset);
  for (int rr = threadIdx.y; rr < t.nrow; rr += blockDim.y) {
    const int r = t.row0 + rr;
    int oslot, bslot;
    const int64_t ovol = csr_vol(fr, out_vol[r], k, oslot);
    const int64_t bvol = csr_vol(fr, base_vol[r], k, bslot);
    double* op = ob + oslot * arrU + ovol * U;
    const double* bp = ib + bslot * arrU + bvol * U;
    const int q0 = row_ptr[r], q1 = row_ptr[r + 1];
    for (int u = threadIdx.x; u < U; u += blockDim.x) {
      if (SPLIT && INTERP) {
        const double base = __ldg(bp + u);
        const F2 b = split_f64(base);
        float acc = 0.f;
        bool only_base = true;
        for (int q = q0; q < q1; ++q) {
          int s;
          const int64_t v = csr_vol(fr, col[q], k, s);
          const double* src = ib + s * arrU + v * U + u;
          if (src == bp + u) continue;  // the base contributes no difference
          only_base = false;
          const F2 x = split_f64(__ldg(src));
          acc = __fmaf_rn(val_f[q], __fadd_rn(__fsub_rn(x.hi, b.hi), __fsub_rn(x.lo, b.lo)), acc);
        }
        op[u] = only_base ? base : add_back(b, acc);
      } else {
        double acc = 0.0;
        for (int q = q0; q < q1; ++q) {
          int s;
          const int64_t v = csr_vol(fr, col[q], k, s);
          acc = fma(val[q], __ldg(ib + s * arrU + v * U + u), acc);
        }
        op[u] = acc;
      }
    }
  }
}

}  // namespace amr
