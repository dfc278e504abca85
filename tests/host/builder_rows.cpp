// Test harness (CPU): prints the explicit operator rows the host builder
// derives for one subface of face 0, as "out col weight" lines with face-0
// flat volume indices, so that a test can compare them with the oracle.
//   builder_rows interp  p k order sub scheme   rows of P (interpolation_rows)
//   builder_rows restrict p k order sub scheme  rows of R (restriction_rows)
//   builder_rows lsclass p k order sub          rows of P rebuilt from the
//       least-squares class tables the interpolation kernel applies (slot
//       layout of ls_interp_core)
//   builder_rows tiles p k order sub precision U budget
//       the interpolation tiles of one item (face 0) as "seg a0 na b0 nb u0
//       nu region_volumes" lines, then "smem <bytes the launch provides>"
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "../../paper_2504_15814_gb300/csrc/builder.hpp"

using namespace amr;

static int P, K;
static long flat(int j, int a, int b) { return ((long)b * P + a) * (2 * K) + (j + K); }  // face 0: x = normal

static void print_rows(const Rows& r) {
  for (size_t i = 0; i < r.rows.size(); ++i) {
    const uint32_t o = r.out_vol[i];
    const long out = ((long)((o >> 6) & 63) * P + (o & 63)) * (2 * K) + ((o >> 12) & 7);
    for (auto& [v, w] : r.rows[i])
      std::printf("%ld %ld %.17g\n", out, ((long)((v >> 6) & 63) * P + (v & 63)) * (2 * K) + ((v >> 12) & 7), w);
  }
}

static void ls_class_rows(int M, int sub) {
  amr_transfer_item it{0, -1, P, K, M, 1, 0, 0};
  amr_transfer_desc d{};
  d.abi_version = AMR_TRANSFER_ABI_VERSION;
  d.num_unknowns = 1;
  d.num_items = 1;
  d.items = &it;
  d.coarse_elems = 2LL * K * P * P;
  d.fine_elems = 9 * d.coarse_elems;
  const LsTables lt = build_ls_tables(d);
  const double* blk = lt.wd.data() + lt.item_off[0];
  std::vector<std::array<int, 3>> alphas;
  for (int x = 0; x <= M; ++x)
    for (int y = 0; x + y <= M; ++y)
      for (int z = 0; x + y + z <= M; ++z)
        if (x + y + z > 0) alphas.push_back({x, y, z});
  const int s0 = sub % 3, s1 = sub / 3;
  for (int i = -1; i >= -K; --i)
    for (int q1 = 0; q1 < P; ++q1)
      for (int q0 = 0; q0 < P; ++q0) {
        const int g0 = s0 * P + q0, g1 = s1 * P + q1, a = g0 / 3, b = g1 / 3;
        const int e[3] = {i + 2, g0 - 3 * a - 1, g1 - 3 * b - 1};
        const double* W = blk + (ls_class(a, P) + 5 * ls_class(b, P)) * LS_SLOTS * LS_NALPHA;
        const int c[3] = {-1, a, b}, lo[3] = {-K, 0, 0}, hi[3] = {K - 1, P - 1, P - 1};
        int ps[3], pl[3], ms[3], ml[3];
        for (int dd = 0; dd < 3; ++dd) {
          stencil_window(c[dd], lo[dd], hi[dd], pure_exactness(M), ps[dd], pl[dd]);
          stencil_window(c[dd], lo[dd], hi[dd], mixed_exactness(M), ms[dd], ml[dd]);
        }
        auto slot_weight = [&](int slot) {
          double w = 0;
          for (size_t al = 0; al < alphas.size(); ++al) {
            double mono = 1;
            for (int dd = 0; dd < 3; ++dd)
              for (int r = 0; r < alphas[al][dd]; ++r) mono *= e[dd];
            w += W[slot * LS_NALPHA + al] * mono;
          }
          return w;
        };
        std::map<long, double> row;
        double total = 0;
        for (int dd = 0; dd < 3; ++dd)
          for (int q = 0; q < pl[dd]; ++q) {
            int x[3] = {c[0], c[1], c[2]};
            x[dd] = ps[dd] + q;
            const double w = slot_weight(dd * 5 + q);
            row[flat(x[0], x[1], x[2])] += w;
            total += w;
          }
        for (int q = 0; q < 3; ++q)
          for (int j = 0; j < 3; ++j)
            for (int ii = 0; ii < 3; ++ii) {
              const double w = slot_weight(15 + (q * 3 + j) * 3 + ii);
              row[flat(ms[0] + ii, ms[1] + j, ms[2] + q)] += w;
              total += w;
            }
        row[flat(-1, a, b)] += 1.0 - total;
        const long out = ((long)q1 * P + q0) * (2 * K) + (i + K);
        for (auto& [col, w] : row)
          if (w != 0) std::printf("%ld %ld %.17g\n", out, col, w);
      }
}

static void tiles(int M, int sub, int precision, int U, int budget) {
  amr_transfer_item it{0, sub, P, K, M, 0, 0, 0};
  amr_transfer_desc d{};
  d.abi_version = AMR_TRANSFER_ABI_VERSION;
  d.num_unknowns = U;
  d.precision = precision;
  d.num_items = 1;
  d.items = &it;
  d.coarse_elems = 2LL * K * P * P * U;
  d.fine_elems = 9 * d.coarse_elems;
  const BuildResult br = build_plan(d, budget, 32);
  if (br.status != AMR_OK) {
    std::printf("error %s\n", br.message.c_str());
    return;
  }
  int64_t seg_end[4], acc = 0;
  for (int q = 0; q < 4; ++q) seg_end[q] = (acc += br.interp_segments[q]);
  for (size_t i = 0; i < br.interp_tiles.size(); ++i) {
    const Tile& t = br.interp_tiles[i];
    int seg = 0;
    while ((int64_t)i >= seg_end[seg]) ++seg;
    IRange rn, ra, rb;
    interp_region(P, K, M, t.a0, t.na, t.b0, t.nb, rn, ra, rb);
    const long vols = (long)(rn.hi - rn.lo + 1) * (ra.hi - ra.lo + 1) * (rb.hi - rb.lo + 1);
    std::printf("%d %d %d %d %d %d %d %ld\n", seg, t.a0, t.na, t.b0, t.nb, t.u0, t.nu, vols);
  }
  std::printf("smem %d\n", br.max_interp_smem);
}

int main(int argc, char** argv) {
  if (argc < 6) return 2;
  P = std::atoi(argv[2]);
  K = std::atoi(argv[3]);
  const int M = std::atoi(argv[4]), sub = std::atoi(argv[5]), scheme = argc > 6 ? std::atoi(argv[6]) : 0;
  if (!std::strcmp(argv[1], "interp")) print_rows(interpolation_rows(sub, 0, P, K, M, scheme));
  else if (!std::strcmp(argv[1], "restrict")) print_rows(restriction_rows(sub, 0, P, K, M, scheme));
  else if (!std::strcmp(argv[1], "lsclass")) ls_class_rows(M, sub);
  else if (!std::strcmp(argv[1], "tiles") && argc > 8) tiles(M, sub, std::atoi(argv[6]), std::atoi(argv[7]), std::atoi(argv[8]));
  else return 2;
  return 0;
}
