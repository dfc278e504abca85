/*
 * amr_transfer.h - C ABI of the GB300 coarse<->fine AMR transfer library.
 *
 * Operation (arXiv 2504.15814, Sec. 2): along a resolution transition of a
 * three-partitioned, 2:1-balanced spacetree, a hanging face separates one
 * coarse patch (p^3 volumes) from 3 x 3 fine patches.  The fine ghost
 * volumes are interpolated from the coarse face data, Q^f = P Q^c, and the
 * coarse halo volumes are restricted from the fine face data, Q^c = R Q^f.
 * The higher-order operators (Sec. 3) reconstruct each output by a Taylor
 * expansion of order 2 or 3 about the nearest input cell centre, with
 * derivatives from finite-difference stencils over neighbouring centres; the
 * d-linear operators are the tensor-product interpolation and averaging
 * restriction of Sec. 2.  Every unknown of a volume uses the same operator
 * (Sec. 2), so the library vectorises over the unknowns of the AoS layout.
 *
 * Data layout (Sec. 4.1: AoS, lexicographic):
 *   A face array holds 2k layers along the face normal (k = overlap / halo
 *   depth on each side) times p x p volumes, lexicographic with x fastest,
 *   and the U unknowns of a volume contiguous (float64).  Face f in 0..5 has
 *   normal axis f % 3; its tangential axes t0 < t1 are the other two.  For
 *   f < 3 the coarse patch lies on the low side of the interface, for f >= 3
 *   on the high side.  Normal index i sits at (i - k + 1/2) * spacing from the
 *   interface.  Subface s = s0 + 3 s1 (s0 along t0, s1 along t1) is the fine
 *   patch covering coarse tangential indices [s_t p/3, (s_t+1) p/3).
 *
 * Ownership: every data buffer is owned by the caller and lies in memory the
 * device can access -- device memory, or pinned (page-locked) host memory,
 * which the kernels then read and write in place; the plan owns its device
 * tables.  All calls that take a stream are
 * asynchronous on that stream (NULL = the legacy default stream); argument
 * errors are detected on the host before anything is enqueued, and then
 * nothing is enqueued.  A plan is bound to the device that was current when
 * it was created and must be used from that device.  A plan may be used by
 * one host thread at a time.
 */
#ifndef AMR_TRANSFER_H
#define AMR_TRANSFER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMR_TRANSFER_ABI_VERSION 1

/* Plan flag: apply every item's operator as explicit sparse rows (CSR, the
 * paper's own storage, Sec. 4.2) instead of the factorised kernels.  Items
 * with scheme 1 always use the sparse rows. */
#define AMR_FLAG_CSR 1

typedef enum {
  AMR_OK = 0,
  AMR_ERR_INVALID_ARGUMENT = 1, /* null pointer, out-of-range field, overlapping outputs */
  AMR_ERR_UNSUPPORTED = 2,      /* valid request this version cannot serve (see item rules) */
  AMR_ERR_OUT_OF_MEMORY = 3,    /* a device or host allocation of the plan failed */
  AMR_ERR_CUDA = 4,             /* a CUDA runtime call failed; the CUDA error is kept */
  AMR_ERR_TIMEOUT = 5,          /* reserved: a bounded device-side wait gave up */
  AMR_ERR_INTERNAL = 6
} amr_status;

typedef enum {
  AMR_ORDER_DLINEAR = 1, /* Sec. 2: d-linear tensor-product interpolation / averaging restriction */
  AMR_ORDER_TAYLOR2 = 2, /* Sec. 3: second-order Taylor, n = 10 coefficients */
  AMR_ORDER_TAYLOR3 = 3  /* Sec. 3: third-order Taylor, n = 20 coefficients */
} amr_order;

typedef enum {
  /* float64 arithmetic throughout; matches the float64 oracle to 1e-12 */
  AMR_PREC_FP64 = 0,
  /* float64 base value u_c and float64-accurate stencil differences
     u_j - u_c; derivative and Taylor-increment arithmetic in float32 on those
     differences; the increment is added back to the float64 base.  Results
     are float64.  The error is a few float32 roundings of the increment:
     about 2^-22 times the largest |child - u_c| of a face, i.e. up to ~1e-6
     of the field's magnitude on fields that vary by O(1) over one coarse
     cell.  Taylor restriction keeps float64 accuracy (~1e-14).  Inputs must
     lie in the float range: magnitudes below 2^-126 are taken as zero,
     magnitudes of 2^128 and more give non-finite results (the injected,
     coincident children excepted), a NaN propagates as NaN. */
  AMR_PREC_SPLIT = 1,
  /* Exact fixed point.  Per interpolation tile and unknown, every staged
     coarse value is rounded once to an integer multiple of q = 3^g 2^-s, the
     grid on which |value / q| < 2^47 for the largest magnitude of that
     unknown in the tile's stencil region (g = 4, 2, 3 for Taylor-3, Taylor-2,
     d-linear); differences, derivatives and the Taylor (or d-linear)
     evaluation then run in exact int64 arithmetic, and each result is rounded
     once to float64.  Error: at most (sum of |weights|) * q / 2, below 1e-13
     of the region's largest magnitude; matches the float64 oracle to 1e-12
     normwise.  Injected (coincident) children are copied exactly.  A region
     holding a NaN or an infinity makes every other child of that unknown in
     the tile NaN; results beyond the float64 range become infinite, below
     its normal range +0; regions whose largest magnitude is below 2^-960
     are quantized on the grid of 2^-960 instead.  Restriction: float64
     for half the coarse columns, exact integer sums on a 62-bit grid per
     column for the other half (float64 accuracy or better).  The
     least-squares scheme uses the float64 kernels. */
  AMR_PREC_FIXED = 2
} amr_precision;

/* One transfer item: one subface (one fine patch, a 1/9 block of P and R,
 * Sec. 2) or a whole hanging face (all nine subfaces). */
typedef struct {
  int32_t face;          /* 0..5, see the layout note above */
  int32_t subface;       /* 0..8 = s0 + 3 s1, or -1 for all nine subfaces */
  int32_t patch_size;    /* p: 1..48 (at least m+1 for Taylor-m).  Coarse volume a covers fine
                            global tangential indices 3a..3a+2 and coincides with 3a+1; for p
                            not a multiple of 3 (Sec. 5.3 notes multiples align better) a
                            subface boundary can cut a coarse volume, which the subface holding
                            3a+1 restricts (d-linear: injected along the cut axis) */
  int32_t overlap;       /* k: 1..5; Taylor-m needs 2k >= m+1 and p >= m+1.  Fine ghost layer
                            -1-g lies inside coarse layer -1-g/3, so k = 4, 5 interpolate the
                            ghost layers -4..-k from a second layer of coarse centres (layer
                            -2); coarse halo layer j >= 1 is extrapolated from fine layer k-1
                            by (3j+2-k) h (an injection where that is 0).  k = 4, 5 need p a
                            multiple of 3 and scheme 0, no AMR_FLAG_CSR, and are served by
                            interpolate and restrict (the adjoint and increment calls return
                            AMR_ERR_UNSUPPORTED for such plans) */
  int32_t order;         /* amr_order */
  int32_t scheme;        /* Taylor derivative estimate: 0 tensor finite-difference stencils (default),
                            1 least-squares polynomial fit through the same centres, constrained
                            through the centre value (Sec. 3: A x = Q^c); must be 0 for d-linear */
  int64_t coarse_offset; /* element (float64) offset of the coarse face array, 2k p^2 U elements */
  int64_t fine_offset;   /* element offset of the fine face array of the subface; for subface -1,
                            nine consecutive fine face arrays in the order s = 0..8 */
} amr_transfer_item;

typedef struct {
  int32_t abi_version;   /* AMR_TRANSFER_ABI_VERSION */
  int32_t num_unknowns;  /* U >= 1: unknowns per volume (58 for first-order CCZ4, Sec. 2) */
  int32_t precision;     /* amr_precision */
  int32_t flags;         /* 0, or AMR_FLAG_CSR */
  int64_t num_items;     /* >= 0 */
  const amr_transfer_item* items; /* host array of num_items; copied at create */
  int64_t coarse_elems;  /* float64 elements of the coarse buffer; every coarse face array must fit */
  int64_t fine_elems;    /* float64 elements of the fine buffer; every fine face array must fit */
} amr_transfer_desc;

typedef struct amr_transfer_plan amr_transfer_plan; /* opaque, owned by the library */

/* Validate the items, build the operator tables and the device work list
 * (Sec. 3: operators are constructed once, off the time-step loop).
 * Rules: fine face arrays of different items must not overlap; items that
 * name the same coarse_offset must agree on face, p and k and own disjoint
 * subfaces; coarse face arrays with different offsets must not overlap.
 * Returns AMR_OK and *out, or an error and *out = NULL. */
amr_status amr_transfer_plan_create(const amr_transfer_desc* desc, amr_transfer_plan** out);

/* Q^f = P Q^c (Sec. 2): writes only the fine ghost halves (the k fine layers
 * on the coarse side) of every item's fine face arrays.  coarse and fine
 * point to coarse_elems / fine_elems float64 values in memory the device can
 * access: device memory, or pinned host memory, which the kernels then read
 * and write in place over the host link (same results, bit for bit); they
 * must not overlap.  The same holds for every buffer of the calls below. */
amr_status amr_transfer_plan_interpolate(amr_transfer_plan* plan, const double* coarse,
                                         double* fine, void* cuda_stream);

/* Q^c = R Q^f (Sec. 2, one call per subface in the paper's appendix "Code
 * Overview"): writes only the coarse halo volumes (the k coarse layers on the
 * fine side) that lie over each item's subfaces.  Reads both halves of the
 * fine face arrays, the ghost half included. */
amr_status amr_transfer_plan_restrict(amr_transfer_plan* plan, const double* fine,
                                      double* coarse, void* cuda_stream);

/* g_coarse = P^T g_fine over the whole coarse buffer: overwrites all
 * coarse_elems values (zero where no weight reaches) and sums the
 * contributions of items that share a coarse face array.  Only the ghost
 * entries of g_fine are read.  Float64 results for every plan precision:
 * groups of items sharing a coarse array whose items all use
 * finite-difference stencils with p a multiple of 3 run the factorised
 * transpose in exact fixed point (the ghost gradients of the group rounded
 * once onto a grid of 2^-44 of their largest magnitude per unknown, then
 * exact integer sums; a group holding a NaN or an infinity gives NaN for that
 * unknown); the other items use explicit transposed rows in float64.  The
 * first adjoint call on a plan builds its transposed-operator tables (host
 * work and a synchronous upload): make it before capturing a stream.
 * AMR_ERR_UNSUPPORTED for plans with an item of overlap 4 or 5. */
amr_status amr_transfer_plan_interpolate_adjoint(amr_transfer_plan* plan, const double* g_fine,
                                                 double* g_coarse, void* cuda_stream);

/* g_fine = R^T g_coarse over the whole fine buffer: overwrites all
 * fine_elems values (zero where no weight reaches).  Only the entries of
 * g_coarse that restriction writes are read.  Float64 arithmetic.
 * AMR_ERR_UNSUPPORTED for plans with an item of overlap 4 or 5. */
amr_status amr_transfer_plan_restrict_adjoint(amr_transfer_plan* plan, const double* g_coarse,
                                              double* g_fine, void* cuda_stream);

/* Split precision with float32 storage of the increments.  For every fine
 * ghost volume and unknown, writes increment = (interpolated value) - (value
 * of the coarse centre nearest to it) as float32, computed exactly as in
 * AMR_PREC_SPLIT (float64-accurate differences, float32 derivative and
 * Taylor arithmetic); coincident volumes get 0.  Layout: item i's increments
 * start at the sum over earlier items of (number of fine face arrays) * k *
 * p^2 * U; inside an item, element (((s * k + g) * p + q1) * p + q0) * U + u
 * for fine face array s, ghost layer g (0 next to the interface), tangential
 * indices q1 (t1) and q0 (t0), unknown u.  increments holds
 * amr_transfer_plan_info.increment_elems floats; d-linear items are included
 * the same way.  Works for plans of either precision; AMR_ERR_UNSUPPORTED for
 * plans with items on the sparse-row path (scheme 1 or AMR_FLAG_CSR) or of
 * overlap 4 or 5. */
amr_status amr_transfer_plan_interpolate_increments(amr_transfer_plan* plan, const double* coarse,
                                                    float* increments, void* cuda_stream);

/* fine ghost value = coarse centre value + increment (float64 result), for
 * the increments written by amr_transfer_plan_interpolate_increments from the
 * same coarse buffer: writes the same fine entries as interpolate. */
amr_status amr_transfer_plan_apply_increments(amr_transfer_plan* plan, const double* coarse,
                                              const float* increments, double* fine, void* cuda_stream);

/* Diagonal (edge and vertex) ghost volumes.  The paper's transfer carries no
 * diagonal data (Sec. 2: only the face arrays of a hanging face); a fine patch
 * whose stencils reach across its edges also needs ghost volumes beyond its
 * subface.  This call fills, for every fine face array of every item, the
 * ghost half widened by k volumes on each tangential side, by the same rule as
 * interpolate: each volume is reconstructed about its nearest coarse centre of
 * the item's coarse face array (the face's edge centre for volumes past the
 * edge, at offsets beyond one fine spacing) with that centre's derivative
 * stencils and Taylor's formula, or by the d-linear tensor product with linear
 * extrapolation past the edge.  Inside the subface the values equal the
 * ordinary ghost values (to rounding).  Float64 arithmetic in every precision
 * mode.  Layout of diag: item i starts at the sum over earlier items of
 * (number of fine face arrays) * k * (p + 2k)^2 * U; inside an item, element
 * ((((s * k + g) * W + q1 + k) * W + q0 + k) * U + u with W = p + 2k, fine
 * face array s, ghost layer g (0 next to the interface), tangential local
 * indices q1 (t1) and q0 (t0) in [-k, p + k), unknown u.  diag_elems is the
 * caller's buffer size; smaller than that sum: AMR_ERR_INVALID_ARGUMENT.
 * Overlaps 1..3 and finite-difference Taylor or d-linear items only
 * (AMR_ERR_UNSUPPORTED otherwise).  The first call on a plan builds its tile
 * table (a synchronous upload): make it before capturing a stream. */
amr_status amr_transfer_plan_interpolate_diagonal(amr_transfer_plan* plan, const double* coarse, double* diag,
                                                  int64_t diag_elems, void* cuda_stream);

/* Plan facts used to report throughput. */
typedef struct {
  int64_t num_items;
  int64_t interp_outputs;      /* fine ghost volumes written by interpolate */
  int64_t restrict_outputs;    /* coarse halo volumes written by restrict */
  int64_t interp_bytes;        /* algorithmic bytes of one interpolate: (volumes referenced by a
                                  non-zero weight + volumes written) * U * 8 */
  int64_t restrict_bytes;      /* the same for one restrict */
  int32_t interp_launches;     /* kernels one interpolate call enqueues */
  int32_t restrict_launches;   /* kernels one restrict call enqueues */
  int64_t increment_elems;     /* float32 values of the increment array (see _interpolate_increments) */
} amr_transfer_plan_info;

amr_status amr_transfer_plan_get_info(const amr_transfer_plan* plan, amr_transfer_plan_info* info);

/* Launch shapes of a plan.  interp_threads: CTA size of the interpolation
 * kernel (a multiple of 32; up to 384 in split precision, 256 in float64);
 * restrict_threads: CTA size of the restriction kernel (32..256, a multiple
 * of 32); interp_smem_budget: bytes of shared memory an interpolation tile
 * may stage (4096..200704; it sets how many unknowns one tile carries);
 * interp_addback (split precision only, 0..3): share of the interpolated
 * children whose float64 result is formed by one float64 add instead of
 * float32 TwoSum + integer assembly -- 0 none, 1 four ninths, 2 two thirds
 * (default), 3 eight ninths; interp_lanes: how interpolation threads map to
 * (coarse centre, unknown) tasks -- 0 packs them densely with the unknown
 * fastest (default), 32 gives every coarse centre one warp whose lanes are
 * its unknowns (a tile then carries at most 32 unknowns), so that a warp
 * never straddles two centres. */
typedef struct {
  int32_t interp_threads;
  int32_t interp_smem_budget;
  int32_t restrict_threads;
  int32_t interp_addback;
  int32_t interp_lanes;
} amr_transfer_tuning;

amr_status amr_transfer_plan_get_tuning(const amr_transfer_plan* plan, amr_transfer_tuning* out);

/* Rebuild the plan's tiles for these launch shapes (synchronous).  Drops a
 * captured step graph. */
amr_status amr_transfer_plan_set_tuning(amr_transfer_plan* plan, const amr_transfer_tuning* tuning);

/* Autotuner: times candidate launch shapes of interpolate and restrict on the
 * caller's buffers (CUDA events on the stream; synchronises it), keeps the
 * fastest, and reports it in *chosen (may be NULL).  fine's ghost halves and
 * coarse_out's restricted halo volumes are overwritten with valid results;
 * coarse_out may equal coarse.  Drops a captured step graph. */
amr_status amr_transfer_plan_autotune(amr_transfer_plan* plan, const double* coarse, double* fine,
                                      double* coarse_out, void* cuda_stream, amr_transfer_tuning* chosen);

/* Capture one transfer step -- interpolate(coarse -> fine) followed by
 * restrict(fine -> coarse_out) -- into a CUDA graph owned by the plan, for
 * these fixed buffers (replaces a previous capture).  Nothing runs until
 * amr_transfer_plan_launch_step.  Not to be called while the caller's
 * stream is itself being captured. */
amr_status amr_transfer_plan_capture_step(amr_transfer_plan* plan, const double* coarse, double* fine,
                                          double* coarse_out);

/* Enqueue the captured step graph on a stream (AMR_ERR_INVALID_ARGUMENT if
 * none is captured). */
amr_status amr_transfer_plan_launch_step(amr_transfer_plan* plan, void* cuda_stream);

/* Release the plan's device tables (synchronises its device).  NULL is a no-op. */
amr_status amr_transfer_plan_destroy(amr_transfer_plan* plan);

/* Static text for a status code; never NULL. */
const char* amr_status_string(amr_status status);

/* Text of the last CUDA error seen by the calling thread in this library
 * (after AMR_ERR_CUDA); never NULL. */
const char* amr_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMR_TRANSFER_H */
