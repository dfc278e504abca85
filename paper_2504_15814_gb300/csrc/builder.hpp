// Host-side operator builder of the transfer library.
//
// The paper constructs the interpolation and restriction operators per call
// and reports that construction dominates the higher-order run time
// (Sec. 5.3); it suggests precomputing them.  This builder does all of it once
// per plan: it validates the items, derives the 1-D derivative weight tables
// from exact rational Lagrange polynomials, cuts the work into tiles, counts
// the algorithmic bytes, and assembles the sparse transposed operators P^T and
// R^T used by the adjoint kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "amr_common.cuh"

namespace amr {

struct Tables {
  double wt_interp[WT_SIZE];  // lambda / (r! 3^r): coefficients in units of the fine spacing
  double wt_restrict[WT_SIZE];  // lambda / r!: coefficients in units of the fine spacing
  float wt_interp_f[WT_SIZE];
  float wt_restrict_f[WT_SIZE];
  double ls[LS_SIZE];
  float ls_f[LS_SIZE];
  double rw[RW_SIZE];     // combined restriction weights
  float rw_hi[RW_SIZE];   // float pair of the same: rw = rw_hi + rw_lo (+ O(2^-48))
  float rw_lo[RW_SIZE];
};

// Built once per process.
const Tables& tables();

// Sparse transposed operator of one face class, in the reference frame.
// Row r = reference volume of the operator's input face array
//   (j + k) * p * p + b * p + a;
// column = slot * (2 k p^2) + reference volume of the output face array.
struct CsrT {
  std::vector<int32_t> row_ptr;  // rows + 1
  std::vector<int32_t> col;
  std::vector<double> val;
};

struct BuildResult {
  amr_status status = AMR_OK;
  std::string message;
  std::vector<Tile> interp_tiles, restrict_tiles;
  int64_t interp_outputs = 0, restrict_outputs = 0;
  int64_t interp_bytes = 0, restrict_bytes = 0;
  int max_interp_smem = 0;  // bytes of dynamic shared memory the interpolation kernel needs
};

BuildResult build_plan(const amr_transfer_desc& desc, int smem_budget);

// Explicit operator rows of P (interpolation) or R (restriction) for one
// subface, in the reference frame: out_vol[i] is the reference volume of the
// output face array, rows[i] the (input reference volume, weight) pairs.
struct Rows {
  std::vector<int32_t> out_vol;
  std::vector<std::vector<std::pair<int32_t, double>>> rows;
};
Rows interpolation_rows(int sub, int p, int k, int order);
Rows restriction_rows(int sub, int p, int k, int order);

}  // namespace amr
