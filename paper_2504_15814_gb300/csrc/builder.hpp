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
  // exact integer numerators of the same Taylor-coefficient weights (lambda / r!,
  // units of the coarse spacing): lambda / r! * fixed_den(L, r), fixed_den = 2
  // for 3-point windows and 12, 24, 12 (r = 1, 2, 3) for 4- and 5-point windows
  int32_t fxw[WT_SIZE];
  // combined restriction weights of the finite-difference scheme as integers
  // rwx = rw * D over the row's denominator D = 2^a 3^b (b <= 1); rw_den per
  // row (index rw_index / 5): a | b << 4
  int32_t rwx[RW_SIZE];
  int32_t rw_den[RW_SIZE / 5];
  // d-linear restriction: least-squares line weights / 9 as integers over a
  // per-row denominator D = 2^a 3^b; ls_den[(k - 1) * kMaxOverlap + j] =
  // a | b << 4 | 1 << 8 (0: no such form, float64 only)
  int32_t lsx[LS_SIZE];
  int32_t ls_den[kMaxOverlap * kMaxOverlap];
};

// Built once per process.
const Tables& tables();

// Packed reference-frame volume of a face array: signed normal layer l
// (stored as l + k, 3 bits), tangential q1 and q0 (6 bits each), and the
// index of the fine face array within the item (4 bits).
__host__ __device__ inline uint32_t pack_vol(int slot, int layer_plus_k, int q1, int q0) {
  return ((uint32_t)slot << 15) | ((uint32_t)layer_plus_k << 12) | ((uint32_t)q1 << 6) | (uint32_t)q0;
}

// Transposed operator (P^T or R^T) of one face class in CSR form.  Row r is
// the reference volume (l + k) p^2 + q1 p + q0 of the adjoint's output face
// array (the coarse array for P^T, the fine array of one subface for R^T);
// entries are packed volumes of the adjoint's input and their weights.
struct CsrT {
  std::vector<int32_t> row_ptr;
  std::vector<uint32_t> col;
  std::vector<double> val;
};

// Explicit operator rows of one subface in the reference frame:
// out_vol[i] (packed) <- sum_e w_e in_vol[e] (packed).
struct Rows {
  std::vector<uint32_t> out_vol;
  std::vector<std::vector<std::pair<uint32_t, double>>> rows;
};
Rows interpolation_rows(int sub, int slot, int p, int k, int order, int scheme = 0);
Rows restriction_rows(int sub, int slot, int p, int k, int order, int scheme = 0);

// Forward sparse rows of the items routed to the CSR kernels (scheme 1, or
// every item with AMR_FLAG_CSR), per face class, for P and for R: row r of a
// class writes out_vol[r] from sum_e val[e] in[col[e]]; base_vol[r] is the
// input volume the split path takes differences against (the nearest input
// centre).
struct CsrFwd {
  std::vector<int32_t> row_ptr;  // absolute into col / val
  std::vector<uint32_t> col, out_vol, base_vol;
  std::vector<double> val;
};
struct CsrTile {
  int32_t item;
  int32_t row0, nrow;  // absolute rows of the concatenated class tables
  int16_t u0, nu;
};
struct CsrBuild {
  CsrFwd pf, rf;                       // interpolation and restriction rows
  std::vector<CsrTile> ptiles, rtiles;
  std::vector<char> routed;            // per item: 1 if it uses the CSR kernels
  int64_t p_nnz = 0, r_nnz = 0;
};
CsrBuild build_csr(const amr_transfer_desc& desc);

// Least-squares derivative tables of the scheme-1 items that the factorised
// interpolation kernel serves: one block of LS_BLOCK weights per distinct
// (p, k, order), layout [class][slot][alpha] then [class][alpha] (column
// sums); alpha / (alpha! 3^|alpha|) scaling folded in (Taylor coefficients in
// units of the fine spacing, like the finite-difference tables).
struct LsTables {
  std::vector<double> wd;
  std::vector<float> wf;
  std::vector<int64_t> item_off;  // per item: offset of its block, or -1
};
LsTables build_ls_tables(const amr_transfer_desc& desc);

struct AdjointTile {
  int32_t index;  // group (P^T) or item (R^T)
  int16_t slot;   // fine face array within the item (R^T)
  int16_t klass;  // class of the item (R^T)
  int16_t u0, nu;
};

struct BuildResult {
  amr_status status = AMR_OK;
  std::string message;
  std::vector<Tile> interp_tiles, restrict_tiles;
  // interp_tiles holds four consecutive segments, counted here: finite
  // differences, then with p not a multiple of 3 (CUT), then least squares,
  // then least squares with CUT
  int64_t interp_segments[4] = {0, 0, 0, 0};
  int64_t interp_outputs = 0, restrict_outputs = 0;
  int64_t interp_bytes = 0, restrict_bytes = 0;
  int max_interp_smem = 0;  // bytes of dynamic shared memory the interpolation kernel needs
  std::vector<int64_t> incr_off;          // float32 increment array offset of each item
  std::vector<AdjointTile> incr_tiles;    // (item, fine face array, unknown chunk) of apply_increments
  int64_t incr_elems = 0;
};

// smem_budget: bytes one interpolation tile may stage; nu_cap: the most
// unknowns one interpolation tile may carry.
BuildResult build_plan(const amr_transfer_desc& desc, int smem_budget, int nu_cap = 32767);

// Adjoint work: P^T over coarse face arrays (items sharing one coarse array
// form a group and are summed in item order), R^T over each item's fine
// face arrays.  Classes are (p, k, order, subface) with subface -1 for a whole
// hanging face.
struct AdjointBuild {
  std::vector<int32_t> group_ptr, group_items, item_class;
  std::vector<AdjointTile> pt_tiles, rt_tiles;  // sparse-row (CSR) work
  // factorised work: P^T of the groups whose items all use finite
  // differences with p a multiple of 3 (fixed-point kernel, 32-unknown
  // chunks, fx_smem bytes of shared memory), R^T of the Taylor items with p a
  // multiple of 3 (one tile per fine face array: item, sub, slot)
  std::vector<AdjointTile> fx_pt_tiles;
  int fx_smem = 0;
  std::vector<Tile> rt_taylor_tiles;
  std::vector<int32_t> cls_pt_rows, cls_rt_rows;  // offset of each class's row_ptr in the concatenation
  CsrT pt, rt;                                    // concatenated classes (row_ptr absolute into col/val)
};
AdjointBuild build_adjoint(const amr_transfer_desc& desc);

}  // namespace amr
