// Host-side operator builder: weight tables, validation, tiling, byte counts.
#include "builder.hpp"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <array>
#include <cmath>
#include <numeric>
#include <set>

namespace amr {
namespace {

// ---------------------------------------------------------------------------
// Exact rational arithmetic for the 1-D weights (small windows: numerators and
// denominators stay far inside int64).
// ---------------------------------------------------------------------------
struct Q {
  int64_t n = 0, d = 1;
  Q() = default;
  Q(int64_t num, int64_t den = 1) : n(num), d(den) { norm(); }
  void norm() {
    if (d < 0) { n = -n; d = -d; }
    int64_t g = std::gcd(n < 0 ? -n : n, d);
    if (g > 1) { n /= g; d /= g; }
  }
  double to_double() const { return (double)n / (double)d; }
};
Q operator+(Q a, Q b) { return Q(a.n * b.d + b.n * a.d, a.d * b.d); }
Q operator-(Q a, Q b) { return Q(a.n * b.d - b.n * a.d, a.d * b.d); }
Q operator*(Q a, Q b) { return Q(a.n * b.n, a.d * b.d); }
Q operator/(Q a, Q b) { return Q(a.n * b.d, a.d * b.n); }

// Coefficient of t^r of the Lagrange basis polynomial l_i(t) on the points
// x_j = j - pos (j = 0..L-1), t measured from the expansion point: equals
// (d^r l_i / dt^r)(0) / r!, i.e. the Taylor coefficient the weight feeds.
Q lagrange_taylor_coeff(int L, int pos, int r, int i) {
  std::vector<Q> poly{Q(1)};
  Q denom(1);
  const int xi = i - pos;
  for (int j = 0; j < L; ++j) {
    if (j == i) continue;
    const int xj = j - pos;
    std::vector<Q> next(poly.size() + 1, Q(0));
    for (size_t q = 0; q < poly.size(); ++q) {  // poly * (t - xj)
      next[q + 1] = next[q + 1] + poly[q];
      next[q] = next[q] - poly[q] * Q(xj);
    }
    poly.swap(next);
    denom = denom * Q(xi - xj);
  }
  if (r >= (int)poly.size()) return Q(0);
  return poly[r] / denom;
}

std::vector<double> ls_taylor_weights(const std::vector<std::array<int, 3>>& rel, int order,
                                      const std::array<long double, 3>& off);

Tables make_tables() {
  Tables t{};
  for (int L = 3; L <= 5; ++L)
    for (int pos = 0; pos < L; ++pos)
      for (int r = 1; r <= 3; ++r) {
        Q scale(1);
        for (int q = 0; q < r; ++q) scale = scale * Q(1, 3);
        for (int i = 0; i < L; ++i) {
          const Q c = lagrange_taylor_coeff(L, pos, r, i);
          const int idx = wt_offset(L) + (pos * 3 + r - 1) * L + i;
          t.wt_restrict[idx] = c.to_double();
          t.wt_interp[idx] = (c * scale).to_double();
          t.wt_restrict_f[idx] = (float)t.wt_restrict[idx];
          t.wt_interp_f[idx] = (float)t.wt_interp[idx];
          const Q n = c * Q(fixed_den(L, r));
          if (n.d != 1) {  // the fixed-point kernels rely on integral numerators
            std::fprintf(stderr, "amr_transfer: non-integral stencil numerator (L %d, pos %d, r %d)\n", L, pos, r);
            std::abort();
          }
          t.fxw[idx] = (int32_t)n.n;
        }
      }
  // Least-squares line through the fine patch's own layers (centres at
  // (i + 1/2)/3 H), evaluated at coarse halo layer j (centre (j + 1/2) H).
  for (int k = 1; k <= kMaxOverlap; ++k) {
    std::vector<int> layers;
    if (k == 1) layers = {-1, 0};
    else for (int i = 0; i < k; ++i) layers.push_back(i);
    const int nl = (int)layers.size();
    Q mean(0);
    for (int i : layers) mean = mean + Q(2 * i + 1, 6);
    mean = mean / Q(nl);
    Q sxx(0);
    for (int i : layers) { Q dx = Q(2 * i + 1, 6) - mean; sxx = sxx + dx * dx; }
    for (int j = 0; j < k; ++j) {
      const Q xc(2 * j + 1, 2);
      Q row[kMaxOverlap];
      for (int s = 0; s < nl; ++s) {
        const Q w = Q(1, nl) + (Q(2 * layers[s] + 1, 6) - mean) * (xc - mean) / sxx;
        t.ls[ls_index(k, j, s)] = w.to_double();
        t.ls_f[ls_index(k, j, s)] = (float)w.to_double();
        row[s] = w / Q(9);  // applied to the sum of the 3 x 3 tangential values
      }
      // exact integer form over D = 2^a 3^b (b <= 3), else marked unusable
      int64_t D = 1;
      for (int s = 0; s < nl; ++s) D = std::lcm(D, row[s].d);
      int a2 = 0, b3 = 0;
      int64_t rest = D;
      while (rest % 2 == 0) { rest /= 2; ++a2; }
      while (rest % 3 == 0) { rest /= 3; ++b3; }
      bool ok = rest == 1 && b3 <= 3 && a2 <= 15;
      for (int s = 0; s < nl && ok; ++s) {
        const Q n = row[s] * Q(D);
        ok = n.d == 1 && n.n < (1 << 10) && n.n > -(1 << 10);
        if (ok) t.lsx[ls_index(k, j, s)] = (int32_t)n.n;
      }
      t.ls_den[(k - 1) * kMaxOverlap + j] = ok ? (a2 | b3 << 4 | 1 << 8) : 0;
    }
  }
  // Combined restriction weights (exact): W[i] = [s + i == k - 1] +
  // sum_r coeff_r(i) e^r with coeff_r the Taylor coefficient weights about
  // fine layer k - 1 on the window (s, L) and e = 3j + 2 - k.
  for (int order = 2; order <= 3; ++order)
    for (int k = 2; k <= kMaxOverlap; ++k)
      for (int j = 1; j < k; ++j) {
        int s0, L;
        stencil_window(k - 1, -k, k - 1, pure_exactness(order), s0, L);
        const int pos = k - 1 - s0;
        const int e = 3 * j + 2 - k;
        Q row[5];
        for (int i = 0; i < 5; ++i) {
          Q w(0);
          if (i < L) {
            if (i == pos) w = w + Q(1);
            Q epow(1);
            for (int r = 1; r <= order; ++r) {
              epow = epow * Q(e);
              w = w + lagrange_taylor_coeff(L, pos, r, i) * epow;
            }
          }
          const int idx = rw_index(order, k, j) + i;
          t.rw[idx] = w.to_double();
          t.rw_hi[idx] = (float)t.rw[idx];
          t.rw_lo[idx] = (float)(t.rw[idx] - (double)t.rw_hi[idx]);
          row[i] = w;
        }
        // exact integer form: D = lcm of the row's denominators = 2^a 3^b
        int64_t D = 1;
        for (int i = 0; i < 5; ++i) D = std::lcm(D, row[i].d);
        int a2 = 0, b3 = 0;
        int64_t rest = D;
        while (rest % 2 == 0) { rest /= 2; ++a2; }
        while (rest % 3 == 0) { rest /= 3; ++b3; }
        if (rest != 1 || b3 > 1 || a2 > 15) {
          std::fprintf(stderr, "amr_transfer: restriction weight denominator %lld (order %d, k %d, j %d)\n",
                       (long long)D, order, k, j);
          std::abort();
        }
        for (int i = 0; i < 5; ++i) {
          const Q n = row[i] * Q(D);
          if (n.d != 1 || n.n >= (1 << 15) || n.n <= -(1 << 15)) {  // the kernel's sums assume |W| < 2^15
            std::fprintf(stderr, "amr_transfer: restriction numerator out of range (order %d, k %d, j %d)\n", order, k, j);
            std::abort();
          }
          t.rwx[rw_index(order, k, j) + i] = (int32_t)n.n;
        }
        t.rw_den[rw_index(order, k, j) / 5] = a2 | b3 << 4;
        // least-squares scheme: the fit along the same window through the
        // expansion value (the base takes 1 - sum of the others)
        std::vector<std::array<int, 3>> rel;
        for (int i = 0; i < L; ++i)
          if (i != pos) rel.push_back({i - pos, 0, 0});
        const std::vector<double> wl = ls_taylor_weights(rel, order, {(long double)e, 0.0L, 0.0L});
        double sum = 0.0;
        for (size_t q = 0; q < rel.size(); ++q) sum += wl[q];
        for (int i = 0; i < 5; ++i) {
          double w = 0.0;
          if (i < L) w = i == pos ? 1.0 - sum : wl[i < pos ? i : i - 1];
          const int idx = rw_index(order, k, j, 1) + i;
          t.rw[idx] = w;
          t.rw_hi[idx] = (float)w;
          t.rw_lo[idx] = (float)(w - (double)t.rw_hi[idx]);
        }
      }
  return t;
}

// Mark the volumes one interpolation centre (cl, a, b) references (kk child
// layers below it); reference volume index (j + k) * p * p + b * p + a.
void mark_interp_layer(std::vector<char>& m, int p, int k, int order, int cl, int kk, int a, int b) {
  auto mark = [&](int j, int aa, int bb) { m[((size_t)(j + k) * p + bb) * p + aa] = 1; };
  if (order == AMR_ORDER_DLINEAR) {
    const int jlo = kk >= 3 ? cl - 1 : cl;
    const int alo = (a == 0) ? 0 : a - 1, ahi = (a == p - 1) ? p - 1 : a + 1;
    const int blo = (b == 0) ? 0 : b - 1, bhi = (b == p - 1) ? p - 1 : b + 1;
    for (int j = jlo; j <= cl + 1; ++j) {
      for (int bb = blo; bb <= bhi; ++bb)
        for (int aa = alo; aa <= ahi; ++aa) mark(j, aa, bb);
    }
    return;
  }
  int s, l;
  const int c[3] = {cl, a, b};
  const int lo[3] = {-k, 0, 0}, hi[3] = {k - 1, p - 1, p - 1};
  for (int d = 0; d < 3; ++d) {  // pure derivatives: lines through the centre
    stencil_window(c[d], lo[d], hi[d], pure_exactness(order), s, l);
    for (int q = s; q < s + l; ++q) {
      int x[3] = {c[0], c[1], c[2]};
      x[d] = q;
      mark(x[0], x[1], x[2]);
    }
  }
  int ms[3], ml[3];
  for (int d = 0; d < 3; ++d) stencil_window(c[d], lo[d], hi[d], mixed_exactness(order), ms[d], ml[d]);
  for (int d = 0; d < 3; ++d)
    for (int e = d + 1; e < 3; ++e)  // mixed pairs: planes
      for (int qd = ms[d]; qd < ms[d] + ml[d]; ++qd)
        for (int qe = ms[e]; qe < ms[e] + ml[e]; ++qe) {
          int x[3] = {c[0], c[1], c[2]};
          x[d] = qd;
          x[e] = qe;
          mark(x[0], x[1], x[2]);
        }
  if (order == 3)  // u_{t0 t1 n}: the box
    for (int q0 = ms[0]; q0 < ms[0] + ml[0]; ++q0)
      for (int q1 = ms[1]; q1 < ms[1] + ml[1]; ++q1)
        for (int q2 = ms[2]; q2 < ms[2] + ml[2]; ++q2) mark(q0, q1, q2);
}

// Every centre layer of tangential position (a, b).
void mark_interp(std::vector<char>& m, int p, int k, int order, int a, int b) {
  for (int ml = 0; ml < centre_layers(k); ++ml) mark_interp_layer(m, p, k, order, -1 - ml, child_layers(k, ml), a, b);
}

// Fine volumes one restriction column references (reference frame of the
// subface's fine array, local tangential q0, q1 of the coincident column).
void mark_restrict(std::vector<char>& m, int p, int k, int order, int q0, int q1) {
  auto mark = [&](int i, int aa, int bb) { m[((size_t)(i + k) * p + bb) * p + aa] = 1; };
  if (order == AMR_ORDER_DLINEAR) {
    // a coarse volume cut by the subface boundary (coincident fine column on
    // the array's edge) is injected along that axis
    const int da0 = (q0 == 0 || q0 == p - 1) ? 0 : 1, db0 = (q1 == 0 || q1 == p - 1) ? 0 : 1;
    const int ilo = (k == 1) ? -1 : 0, ihi = (k == 1) ? 0 : k - 1;
    for (int i = ilo; i <= ihi; ++i)
      for (int db = -db0; db <= db0; ++db)
        for (int da = -da0; da <= da0; ++da) mark(i, q0 + da, q1 + db);
    return;
  }
  if (k >= 2) mark(1, q0, q1);  // injection
  if (k >= 2 && k - 1 >= 1) {
    int s, l;
    stencil_window(k - 1, -k, k - 1, pure_exactness(order), s, l);
    for (int i = s; i < s + l; ++i) mark(i, q0, q1);
  }
}

}  // namespace

const Tables& tables() {
  static const Tables t = make_tables();
  return t;
}

bool csr_routed(const amr_transfer_desc& desc, const amr_transfer_item& x);

static BuildResult fail(amr_status st, const std::string& msg) {
  BuildResult r;
  r.status = st;
  r.message = msg;
  return r;
}

BuildResult build_plan(const amr_transfer_desc& desc, int smem_budget, int nu_cap) {
  if (desc.abi_version != AMR_TRANSFER_ABI_VERSION)
    return fail(AMR_ERR_INVALID_ARGUMENT, "abi_version mismatch");
  if (desc.num_unknowns < 1) return fail(AMR_ERR_INVALID_ARGUMENT, "num_unknowns must be >= 1");
  if (desc.num_unknowns > 32767) return fail(AMR_ERR_UNSUPPORTED, "num_unknowns > 32767");
  if (desc.precision != AMR_PREC_FP64 && desc.precision != AMR_PREC_SPLIT && desc.precision != AMR_PREC_FIXED)
    return fail(AMR_ERR_INVALID_ARGUMENT, "unknown precision");
  if (desc.flags & ~AMR_FLAG_CSR) return fail(AMR_ERR_INVALID_ARGUMENT, "unknown flags");
  if (desc.num_items < 0 || (desc.num_items > 0 && desc.items == nullptr))
    return fail(AMR_ERR_INVALID_ARGUMENT, "bad item list");
  if (desc.num_items > (int64_t)1 << 30) return fail(AMR_ERR_UNSUPPORTED, "too many items");
  if (desc.coarse_elems < 0 || desc.fine_elems < 0) return fail(AMR_ERR_INVALID_ARGUMENT, "negative buffer size");

  const int64_t U = desc.num_unknowns;
  BuildResult r;
  struct Interval { int64_t lo, hi; int64_t item; };
  std::vector<Interval> fine_iv;
  std::map<int64_t, std::vector<int64_t>> coarse_groups;

  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    char buf[160];
    auto bad = [&](amr_status st, const char* what) {
      std::snprintf(buf, sizeof buf, "item %lld: %s", (long long)it, what);
      return fail(st, buf);
    };
    if (x.face < 0 || x.face > 5) return bad(AMR_ERR_INVALID_ARGUMENT, "face not in 0..5");
    if (x.subface < -1 || x.subface > 8) return bad(AMR_ERR_INVALID_ARGUMENT, "subface not in -1..8");
    if (x.order < 1 || x.order > 3) return bad(AMR_ERR_INVALID_ARGUMENT, "order not in 1..3");
    if (x.scheme != 0 && x.scheme != 1) return bad(AMR_ERR_INVALID_ARGUMENT, "scheme not in 0..1");
    if (x.scheme == 1 && x.order == AMR_ORDER_DLINEAR) return bad(AMR_ERR_UNSUPPORTED, "least-squares scheme needs a Taylor order");
    if (x.patch_size < 1 || x.overlap < 1) return bad(AMR_ERR_INVALID_ARGUMENT, "p and k must be positive");
    if (x.overlap > x.patch_size) return bad(AMR_ERR_INVALID_ARGUMENT, "k > p");
    if (x.patch_size > 48) return bad(AMR_ERR_UNSUPPORTED, "p > 48");
    if (x.overlap > kMaxOverlap) return bad(AMR_ERR_UNSUPPORTED, "k > 5");
    if (x.overlap > 3 && (x.patch_size % 3 != 0 || x.scheme != 0 || (desc.flags & AMR_FLAG_CSR)))
      return bad(AMR_ERR_UNSUPPORTED, "k > 3 needs p a multiple of 3, finite-difference derivatives, no CSR flag");
    if (x.order >= 2 && (2 * x.overlap < x.order + 1 || x.patch_size < x.order + 1))
      return bad(AMR_ERR_UNSUPPORTED, "Taylor order needs 2k >= m+1 and p >= m+1");
    if (x.coarse_offset < 0 || x.fine_offset < 0) return bad(AMR_ERR_INVALID_ARGUMENT, "negative offset");
    const int64_t arr = 2LL * x.overlap * x.patch_size * x.patch_size * U;
    const int64_t nsub = x.subface < 0 ? 9 : 1;
    if (x.coarse_offset > desc.coarse_elems - arr) return bad(AMR_ERR_INVALID_ARGUMENT, "coarse face array out of range");
    if (x.fine_offset > desc.fine_elems - nsub * arr) return bad(AMR_ERR_INVALID_ARGUMENT, "fine face arrays out of range");
    fine_iv.push_back({x.fine_offset, x.fine_offset + nsub * arr, it});
    coarse_groups[x.coarse_offset].push_back(it);
  }
  std::sort(fine_iv.begin(), fine_iv.end(), [](const Interval& a, const Interval& b) { return a.lo < b.lo; });
  for (size_t i = 1; i < fine_iv.size(); ++i)
    if (fine_iv[i].lo < fine_iv[i - 1].hi) return fail(AMR_ERR_INVALID_ARGUMENT, "fine face arrays of two items overlap");
  int64_t prev_hi = INT64_MIN;
  for (auto& [off, members] : coarse_groups) {
    const amr_transfer_item& f = desc.items[members[0]];
    int used = 0;
    for (int64_t m : members) {
      const amr_transfer_item& x = desc.items[m];
      if (x.face != f.face || x.patch_size != f.patch_size || x.overlap != f.overlap)
        return fail(AMR_ERR_INVALID_ARGUMENT, "items sharing a coarse face array disagree on face, p or k");
      const int mask = x.subface < 0 ? 0x1ff : (1 << x.subface);
      if (used & mask) return fail(AMR_ERR_INVALID_ARGUMENT, "items sharing a coarse face array restrict the same subface");
      used |= mask;
    }
    if (off < prev_hi) return fail(AMR_ERR_INVALID_ARGUMENT, "coarse face arrays overlap");
    prev_hi = off + 2LL * f.overlap * f.patch_size * f.patch_size * U;
  }

  // Tiles and byte counts.
  const int TMAX = 12;
  // interpolation tiles go to one of four segments, each run by its own
  // kernel variant: patch size a multiple of 3 or not (children of one
  // coarse centre may lie in two fine face arrays), finite-difference or
  // least-squares derivatives
  std::vector<Tile> seg[4];
  auto region_vols = [](int p, int k, int m, int a0, int na, int b0, int nb) {
    IRange rn, ra, rb;
    interp_region(p, k, m, a0, na, b0, nb, rn, ra, rb);
    return (int64_t)(rn.hi - rn.lo + 1) * (ra.hi - ra.lo + 1) * (rb.hi - rb.lo + 1);
  };
  auto add_interp_tiles = [&](int64_t it, int sub, int slot, int alo, int ahi, int blo, int bhi, int p, int k, int m) {
    const bool ls = desc.items[it].scheme == 1;
    std::vector<Tile>& dst = seg[(p % 3 ? 1 : 0) + (ls ? 2 : 0)];
    // the fixed-point kernel stages 32 unknown slots per region volume
    // (lane stride 32); its tiles shrink until the largest region fits the
    // budget (at least one centre per tile)
    const bool fixed = desc.precision == AMR_PREC_FIXED && !ls;
    int ta = std::min(TMAX, ahi - alo), tb = std::min(TMAX, bhi - blo);
    if (fixed) {
      auto worst = [&](int na, int nb) {
        int64_t v = 0;
        for (int a0 = alo; a0 < ahi; a0 += na)
          for (int b0 = blo; b0 < bhi; b0 += nb)
            v = std::max(v, region_vols(p, k, m, a0, std::min(na, ahi - a0), b0, std::min(nb, bhi - b0)));
        return v;
      };
      while ((ta > 1 || tb > 1) && worst(ta, tb) * 32 * 8 > smem_budget) {
        if (ta >= tb) --ta;
        else --tb;
      }
    }
    for (int a0 = alo; a0 < ahi; a0 += ta)
      for (int b0 = blo; b0 < bhi; b0 += tb) {
        const int na = std::min(ta, ahi - a0), nb = std::min(tb, bhi - b0);
        const int64_t vols = region_vols(p, k, m, a0, na, b0, nb);
        const int nu_max =
            fixed ? (int)std::min<int64_t>(U, 32)
                  : (int)std::min<int64_t>(std::min<int64_t>(U, nu_cap), std::max<int64_t>(1, smem_budget / (vols * 8)));
        const int nchunks = (int)((U + nu_max - 1) / nu_max);
        const int nu = (int)((U + nchunks - 1) / nchunks);
        for (int c = 0; c < nchunks; ++c) {
          Tile t{};
          t.item = (int32_t)it; t.sub = (int8_t)sub; t.slot = (int8_t)slot;
          t.na = (int8_t)na; t.nb = (int8_t)nb; t.a0 = (int16_t)a0; t.b0 = (int16_t)b0;
          t.u0 = (int16_t)(c * nu); t.nu = (int16_t)std::min<int64_t>(nu, U - c * nu);
          dst.push_back(t);
          r.max_interp_smem = std::max<int>(r.max_interp_smem, (int)(vols * (fixed ? 32 : t.nu) * 8));
        }
      }
  };
  auto add_restrict_tiles = [&](int64_t it, int sub, int slot, int alo, int ahi, int blo, int bhi) {
    for (int a0 = alo; a0 < ahi; a0 += TMAX)
      for (int b0 = blo; b0 < bhi; b0 += TMAX) {
        Tile t{};
        t.item = (int32_t)it; t.sub = (int8_t)sub; t.slot = (int8_t)slot;
        t.na = (int8_t)std::min(TMAX, ahi - a0); t.nb = (int8_t)std::min(TMAX, bhi - b0);
        t.a0 = (int16_t)a0; t.b0 = (int16_t)b0;
        for (int64_t u0 = 0; u0 < U; u0 += 128) {
          t.u0 = (int16_t)u0; t.nu = (int16_t)std::min<int64_t>(128, U - u0);
          r.restrict_tiles.push_back(t);
        }
      }
  };
  std::map<std::tuple<int, int, int, int>, int64_t> ref_cache;  // (p,k,order,sub) -> restriction references
  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    const int p = x.patch_size, k = x.overlap, m = x.order;
    std::vector<char> cmark((size_t)2 * k * p * p, 0);
    const bool fused = !csr_routed(desc, x);  // factorised kernels (else the CSR kernels)
    if (x.subface < 0 && fused) {
      add_interp_tiles(it, -1, -1, 0, p, 0, p, p, k, m);
      add_restrict_tiles(it, -1, -1, 0, p, 0, p);
    }
    for (int sl = 0; sl < (x.subface < 0 ? 9 : 1); ++sl) {
      const int sub = x.subface < 0 ? sl : x.subface;
      const int s0 = sub % 3, s1 = sub / 3;
      int ca0, ca1, cb0, cb1, oa0, oa1, ob0, ob1;  // covering and owned coarse ranges
      covering_range(s0, p, ca0, ca1);
      covering_range(s1, p, cb0, cb1);
      owned_range(s0, p, oa0, oa1);
      owned_range(s1, p, ob0, ob1);
      if (x.subface >= 0 && fused) add_interp_tiles(it, sub, 0, ca0, ca1, cb0, cb1, p, k, m);
      if (x.subface >= 0 && fused) add_restrict_tiles(it, sub, 0, oa0, oa1, ob0, ob1);
      for (int b = cb0; b < cb1; ++b)
        for (int a = ca0; a < ca1; ++a) mark_interp(cmark, p, k, m, a, b);
      auto key = std::make_tuple(p, k, m, sub);
      auto f = ref_cache.find(key);
      if (f == ref_cache.end()) {
        std::vector<char> fmark((size_t)2 * k * p * p, 0);
        for (int b = ob0; b < ob1; ++b)
          for (int a = oa0; a < oa1; ++a) mark_restrict(fmark, p, k, m, 3 * a + 1 - s0 * p, 3 * b + 1 - s1 * p);
        f = ref_cache.emplace(key, (int64_t)std::count(fmark.begin(), fmark.end(), 1)).first;
      }
      r.restrict_bytes += f->second * U * 8;
      r.interp_outputs += (int64_t)k * p * p;
      r.restrict_outputs += (int64_t)k * (oa1 - oa0) * (ob1 - ob0);
    }
    r.interp_bytes += (int64_t)std::count(cmark.begin(), cmark.end(), 1) * U * 8;
  }
  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    const int nsub = x.subface < 0 ? 9 : 1;
    r.incr_off.push_back(r.incr_elems);
    r.incr_elems += (int64_t)nsub * x.overlap * x.patch_size * x.patch_size * U;
    for (int sl = 0; sl < nsub; ++sl)
      for (int64_t u0 = 0; u0 < U; u0 += 128)
        r.incr_tiles.push_back({(int32_t)it, (int16_t)sl, 0, (int16_t)u0, (int16_t)std::min<int64_t>(128, U - u0)});
  }
  r.interp_bytes += r.interp_outputs * U * 8;
  r.restrict_bytes += r.restrict_outputs * U * 8;
  for (int q = 0; q < 4; ++q) {
    r.interp_segments[q] = (int64_t)seg[q].size();
    r.interp_tiles.insert(r.interp_tiles.end(), seg[q].begin(), seg[q].end());
  }
  return r;
}

}  // namespace amr

// ---------------------------------------------------------------------------
// Explicit operator rows and their transposes (adjoint).
// ---------------------------------------------------------------------------
namespace amr {
namespace {

using Row = std::map<uint32_t, double>;

// 1-D stencil of derivative order r (0 = point evaluation) about c on
// [lo, hi] with exactness degree E: (index, weight) pairs from a table of
// Taylor-coefficient weights.
std::vector<std::pair<int, double>> axis_stencil(const double* wt, int c, int lo, int hi, int E, int r) {
  if (r == 0) return {{c, 1.0}};
  int s, L;
  stencil_window(c, lo, hi, E, s, L);
  std::vector<std::pair<int, double>> out;
  for (int i = 0; i < L; ++i) {
    const double w = wt[wt_offset(L) + ((c - s) * 3 + r - 1) * L + i];
    if (w != 0.0) out.push_back({s + i, w});
  }
  return out;
}

void add_taylor_interp_row(Row& row, int p, int k, int order, int a, int b, int en, int e0, int e1) {
  const double* wt = tables().wt_interp;
  for (int x = 0; x <= order; ++x)
    for (int y = 0; x + y <= order; ++y)
      for (int z = 0; x + y + z <= order; ++z) {
        double coeff = 1.0;
        for (int q = 0; q < x; ++q) coeff *= en;
        for (int q = 0; q < y; ++q) coeff *= e0;
        for (int q = 0; q < z; ++q) coeff *= e1;
        if (coeff == 0.0) continue;
        const int nz = (x > 0) + (y > 0) + (z > 0);
        const int E = nz <= 1 ? pure_exactness(order) : mixed_exactness(order);
        const auto sn = axis_stencil(wt, -1, -k, k - 1, E, x);
        const auto s0 = axis_stencil(wt, a, 0, p - 1, E, y);
        const auto s1 = axis_stencil(wt, b, 0, p - 1, E, z);
        for (auto& [jn, wn] : sn)
          for (auto& [ja, wa] : s0)
            for (auto& [jb, wb] : s1) row[pack_vol(0, jn + k, jb, ja)] += coeff * wn * wa * wb;
      }
}

// d-linear weights along one axis for child offset e in {-1, 0, 1} about
// coarse index c with neighbours available on [0, n-1].
std::vector<std::pair<int, double>> dlin_axis(int c, int n, int e) {
  if (e == 0) return {{c, 1.0}};
  if (e < 0) {
    if (c > 0) return {{c - 1, 1.0 / 3.0}, {c, 2.0 / 3.0}};
    return {{c, 4.0 / 3.0}, {c + 1, -1.0 / 3.0}};
  }
  if (c < n - 1) return {{c, 2.0 / 3.0}, {c + 1, 1.0 / 3.0}};
  return {{c - 1, -1.0 / 3.0}, {c, 4.0 / 3.0}};
}

// Least-squares Taylor weights (scheme 1): for the points `rel` (offsets from
// the expansion centre, grid units, centre excluded), the fitted derivatives
// x = (A^T A)^-1 A^T (u - u_c) with basis r^alpha / alpha!, evaluated in
// Taylor's formula at offset `off`; returns the weight of each point (the
// centre gets 1 - sum).  Derivatives the points carry no information about
// (zero columns) are not fitted; their terms vanish at `off` by construction.
// The derivatives 0 < |alpha| <= order in the order the kernels use.
std::vector<std::array<int, 3>> taylor_alphas(int order) {
  std::vector<std::array<int, 3>> alphas;
  for (int x = 0; x <= order; ++x)
    for (int y = 0; x + y <= order; ++y)
      for (int z = 0; x + y + z <= order; ++z)
        if (x + y + z > 0) alphas.push_back({x, y, z});
  return alphas;
}

long double factorial(int n) {
  long double f = 1;
  for (int q = 2; q <= n; ++q) f *= q;
  return f;
}

// Least-squares fit of the derivatives D^alpha u (unit spacing,
// taylor_alphas order) of the Taylor polynomial through u(c) to the
// differences d_q = u(c + r_q) - u(c) at the points rel: returns coef[a][q]
// with D^alpha u = sum_q coef[a][q] d_q, by the normal equations in long
// double.  Derivatives the points carry no
// information about (zero columns) are not fitted: their rows are zero.
std::vector<std::vector<long double>> ls_fit(const std::vector<std::array<int, 3>>& rel, int order) {
  const std::vector<std::array<int, 3>> alphas = taylor_alphas(order);
  auto basis = [&](const std::array<int, 3>& r, const std::array<int, 3>& a) {
    long double v = 1;
    for (int d = 0; d < 3; ++d) v *= std::pow((long double)r[d], a[d]) / factorial(a[d]);
    return v;
  };
  std::vector<int> used;
  for (size_t a = 0; a < alphas.size(); ++a) {
    bool any = false;
    for (auto& r : rel) any |= basis(r, alphas[a]) != 0;
    if (any) used.push_back((int)a);
  }
  const int n = (int)used.size(), m = (int)rel.size();
  // augmented normal equations [A^T A | A^T]
  std::vector<std::vector<long double>> aug(n, std::vector<long double>(n + m, 0));
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j)
      for (int q = 0; q < m; ++q) aug[i][j] += basis(rel[q], alphas[used[i]]) * basis(rel[q], alphas[used[j]]);
    for (int q = 0; q < m; ++q) aug[i][n + q] = basis(rel[q], alphas[used[i]]);
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(aug[r][col]) > std::fabs(aug[piv][col])) piv = r;
    std::swap(aug[col], aug[piv]);
    const long double inv = 1 / aug[col][col];
    for (auto& v : aug[col]) v *= inv;
    for (int r = 0; r < n; ++r)
      if (r != col && aug[r][col] != 0) {
        const long double f = aug[r][col];
        for (int c = 0; c < n + m; ++c) aug[r][c] -= f * aug[col][c];
      }
  }
  std::vector<std::vector<long double>> coef(alphas.size(), std::vector<long double>(m, 0));
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < m; ++q) coef[used[i]][q] = aug[i][n + q];
  return coef;
}

// Weights of the least-squares Taylor-m reconstruction at offset `off` on the
// points rel (the centre gets 1 - sum).
std::vector<double> ls_taylor_weights(const std::vector<std::array<int, 3>>& rel, int order,
                                      const std::array<long double, 3>& off) {
  const std::vector<std::array<int, 3>> alphas = taylor_alphas(order);
  const std::vector<std::vector<long double>> coef = ls_fit(rel, order);
  std::vector<double> w(rel.size(), 0.0);
  for (size_t a = 0; a < alphas.size(); ++a) {
    long double mono = 1;
    for (int d = 0; d < 3; ++d) mono *= std::pow(off[d], alphas[a][d]) / factorial(alphas[a][d]);
    if (mono == 0) continue;
    for (size_t q = 0; q < rel.size(); ++q) w[q] += (double)(mono * coef[a][q]);
  }
  return w;
}

// Support of the finite-difference stencils of Taylor-m about centre c on
// the index box [lo, hi] (pure lines, mixed planes, and for m = 3 the box).
std::vector<std::array<int, 3>> stencil_support(const int c[3], const int lo[3], const int hi[3], int order) {
  std::set<std::array<int, 3>> pts;
  int s, l;
  for (int d = 0; d < 3; ++d) {
    stencil_window(c[d], lo[d], hi[d], pure_exactness(order), s, l);
    for (int q = s; q < s + l; ++q) {
      std::array<int, 3> x{c[0], c[1], c[2]};
      x[d] = q;
      pts.insert(x);
    }
  }
  int ms[3], ml[3];
  for (int d = 0; d < 3; ++d) stencil_window(c[d], lo[d], hi[d], mixed_exactness(order), ms[d], ml[d]);
  for (int d = 0; d < 3; ++d)
    for (int e = d + 1; e < 3; ++e)
      for (int qd = ms[d]; qd < ms[d] + ml[d]; ++qd)
        for (int qe = ms[e]; qe < ms[e] + ml[e]; ++qe) {
          std::array<int, 3> x{c[0], c[1], c[2]};
          x[d] = qd;
          x[e] = qe;
          pts.insert(x);
        }
  if (order == 3)
    for (int q0 = ms[0]; q0 < ms[0] + ml[0]; ++q0)
      for (int q1 = ms[1]; q1 < ms[1] + ml[1]; ++q1)
        for (int q2 = ms[2]; q2 < ms[2] + ml[2]; ++q2) pts.insert({q0, q1, q2});
  return std::vector<std::array<int, 3>>(pts.begin(), pts.end());
}

}  // namespace

Rows interpolation_rows(int sub, int slot, int p, int k, int order, int scheme) {
  Rows r;
  const int s0 = sub % 3, s1 = sub / 3;
  for (int i = -k; i <= -1; ++i)
    for (int q1 = 0; q1 < p; ++q1)
      for (int q0 = 0; q0 < p; ++q0) {
        const int g0 = s0 * p + q0, g1 = s1 * p + q1;
        const int a = g0 / 3, b = g1 / 3;
        const int e0 = g0 - 3 * a - 1, e1 = g1 - 3 * b - 1, en = i + 2;
        Row row;
        if (order == AMR_ORDER_DLINEAR) {
          std::vector<std::pair<int, double>> wn;
          if (en == 1) wn = {{-1, 2.0 / 3.0}, {0, 1.0 / 3.0}};
          else if (en == 0) wn = {{-1, 1.0}};
          else wn = {{-2, 1.0 / 3.0}, {-1, 2.0 / 3.0}};
          for (auto& [jn, w_n] : wn)
            for (auto& [ja, w_a] : dlin_axis(a, p, e0))
              for (auto& [jb, w_b] : dlin_axis(b, p, e1)) row[pack_vol(0, jn + k, jb, ja)] += w_n * w_a * w_b;
        } else if (scheme == 1) {
          const int c[3] = {-1, a, b}, lo[3] = {-k, 0, 0}, hi[3] = {k - 1, p - 1, p - 1};
          std::vector<std::array<int, 3>> rel;
          for (auto& x : stencil_support(c, lo, hi, order))
            if (x[0] != c[0] || x[1] != c[1] || x[2] != c[2]) rel.push_back({x[0] - c[0], x[1] - c[1], x[2] - c[2]});
          const std::array<long double, 3> off{en / 3.0L, e0 / 3.0L, e1 / 3.0L};
          const std::vector<double> w = ls_taylor_weights(rel, order, off);
          double sum = 0.0;
          for (size_t q = 0; q < rel.size(); ++q) {
            row[pack_vol(0, c[0] + rel[q][0] + k, c[2] + rel[q][2], c[1] + rel[q][1])] += w[q];
            sum += w[q];
          }
          row[pack_vol(0, -1 + k, b, a)] += 1.0 - sum;
        } else {
          add_taylor_interp_row(row, p, k, order, a, b, en, e0, e1);
        }
        r.out_vol.push_back(pack_vol(slot, i + k, q1, q0));
        r.rows.emplace_back(row.begin(), row.end());
      }
  return r;
}

Rows restriction_rows(int sub, int slot, int p, int k, int order, int scheme) {
  Rows r;
  const Tables& t = tables();
  const int s0 = sub % 3, s1 = sub / 3;
  int a_lo, a_hi, b_lo, b_hi;
  owned_range(s0, p, a_lo, a_hi);
  owned_range(s1, p, b_lo, b_hi);
  for (int j = 0; j < k; ++j)
    for (int b = b_lo; b < b_hi; ++b)
      for (int a = a_lo; a < a_hi; ++a) {
        const int q0 = 3 * a + 1 - s0 * p, q1 = 3 * b + 1 - s1 * p;
        Row row;
        if (order == AMR_ORDER_DLINEAR) {
          // tangential: the average of the 3 fine volumes inside the coarse
          // volume, or injection of the coincident one along an axis where
          // the subface boundary cuts the coarse volume
          const int da0 = (q0 == 0 || q0 == p - 1) ? 0 : 1, db0 = (q1 == 0 || q1 == p - 1) ? 0 : 1;
          const double nt = (double)((2 * da0 + 1) * (2 * db0 + 1));
          const int nl = k == 1 ? 2 : k;
          for (int sl = 0; sl < nl; ++sl) {
            const int i = k == 1 ? sl - 1 : sl;
            const double wl = t.ls[ls_index(k, j, sl)] / nt;
            for (int db = -db0; db <= db0; ++db)
              for (int da = -da0; da <= da0; ++da) row[pack_vol(slot, i + k, q1 + db, q0 + da)] += wl;
          }
        } else if (j == 0) {
          row[pack_vol(slot, 1 + k, q1, q0)] = 1.0;
        } else {
          // combined weights of the window about fine layer k - 1 (finite
          // differences, or the least-squares fit along the same window)
          int s, L;
          stencil_window(k - 1, -k, k - 1, pure_exactness(order), s, L);
          for (int i = 0; i < L; ++i) {
            const double wv = t.rw[rw_index(order, k, j, scheme) + i];
            if (wv != 0.0) row[pack_vol(slot, s + i + k, q1, q0)] += wv;
          }
        }
        r.out_vol.push_back(pack_vol(0, j + k, b, a));
        r.rows.emplace_back(row.begin(), row.end());
      }
  return r;
}

namespace {

// Row index of a packed volume in a CSR over nslot face arrays of 2k p^2 volumes.
int row_of(uint32_t v, int p, int k) {
  const int slot = (int)(v >> 15), lk = (int)((v >> 12) & 7), q1 = (int)((v >> 6) & 63), q0 = (int)(v & 63);
  return ((slot * 2 * k + lk) * p + q1) * p + q0;
}

void append_transpose(CsrT& out, std::vector<int32_t>& cls_rows, const std::vector<Rows>& blocks, int nrows, int p,
                      int k) {
  std::vector<std::vector<std::pair<uint32_t, double>>> t(nrows);
  for (const Rows& blk : blocks)
    for (size_t i = 0; i < blk.rows.size(); ++i)
      for (auto& [in_vol, w] : blk.rows[i]) t[row_of(in_vol, p, k)].push_back({blk.out_vol[i], w});
  cls_rows.push_back((int32_t)out.row_ptr.size());
  for (int r = 0; r < nrows; ++r) {
    out.row_ptr.push_back((int32_t)out.col.size());
    for (auto& [c, w] : t[r]) {
      out.col.push_back(c);
      out.val.push_back(w);
    }
  }
  out.row_ptr.push_back((int32_t)out.col.size());
}

}  // namespace

AdjointBuild build_adjoint(const amr_transfer_desc& desc) {
  AdjointBuild ab;
  const int64_t U = desc.num_unknowns;
  std::map<std::tuple<int, int, int, int>, int> classes;
  std::map<int64_t, std::vector<int32_t>> groups;
  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    auto key = std::make_tuple(x.patch_size, x.overlap, x.order * 2 + x.scheme, x.subface);
    auto f = classes.find(key);
    if (f == classes.end()) {
      const int id = (int)classes.size();
      f = classes.emplace(key, id).first;
      const int p = x.patch_size, k = x.overlap, m = x.order;
      std::vector<Rows> pblocks, rblocks;
      const int nsub = x.subface < 0 ? 9 : 1;
      for (int sl = 0; sl < nsub; ++sl) {
        const int sub = x.subface < 0 ? sl : x.subface;
        pblocks.push_back(interpolation_rows(sub, sl, p, k, m, x.scheme));
        rblocks.push_back(restriction_rows(sub, sl, p, k, m, x.scheme));
      }
      const int arr = 2 * k * p * p;
      append_transpose(ab.pt, ab.cls_pt_rows, pblocks, arr, p, k);
      append_transpose(ab.rt, ab.cls_rt_rows, rblocks, nsub * arr, p, k);
    }
    ab.item_class.push_back(f->second);
    groups[x.coarse_offset].push_back((int32_t)it);
  }
  ab.group_ptr.push_back(0);
  const int kFxSmemMax = 112 * 1024;
  for (auto& [off, members] : groups) {
    const int32_t g = (int32_t)ab.group_ptr.size() - 1;
    for (int32_t m : members) ab.group_items.push_back(m);
    ab.group_ptr.push_back((int32_t)ab.group_items.size());
    // factorised fixed-point P^T: finite differences, p a multiple of 3, and
    // an accumulator (union of the normal stencil ranges x p x p x 32 slots)
    // that fits the shared memory of two CTAs per SM
    const amr_transfer_item& f = desc.items[members[0]];
    bool fx = f.patch_size % 3 == 0;
    int rlo = 0, rhi = -1;
    for (int32_t m : members) {
      const amr_transfer_item& x = desc.items[m];
      fx = fx && x.scheme == 0;
      IRange rn, ra, rb;
      interp_region(x.patch_size, x.overlap, x.order, 0, x.patch_size, 0, x.patch_size, rn, ra, rb);
      rlo = std::min(rlo, rn.lo);
      rhi = std::max(rhi, rn.hi);
    }
    const int64_t smem = (int64_t)(rhi - rlo + 1) * f.patch_size * f.patch_size * 32 * 8;
    fx = fx && smem <= kFxSmemMax && !(desc.flags & AMR_FLAG_CSR);
    if (fx) {
      ab.fx_smem = std::max<int>(ab.fx_smem, (int)smem);
      const int nch = (int)((U + 31) / 32), nu = (int)((U + nch - 1) / nch);
      for (int c = 0; c < nch; ++c)
        ab.fx_pt_tiles.push_back({g, 0, 0, (int16_t)(c * nu), (int16_t)std::min<int64_t>(nu, U - c * nu)});
    } else {
      for (int64_t u0 = 0; u0 < U; u0 += 128)
        ab.pt_tiles.push_back({g, 0, 0, (int16_t)u0, (int16_t)std::min<int64_t>(128, U - u0)});
    }
  }
  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    const int nsub = x.subface < 0 ? 9 : 1;
    // direct R^T of Taylor items, p a multiple of 3 (each coarse halo column
    // reaches only its own coincident fine column): one tile per fine face
    // array, which the kernel writes whole
    if (x.order >= 2 && x.patch_size % 3 == 0 && !(desc.flags & AMR_FLAG_CSR)) {
      for (int sl = 0; sl < nsub; ++sl) {
        Tile t{};
        t.item = (int32_t)it;
        t.sub = (int8_t)(x.subface < 0 ? sl : x.subface);
        t.slot = (int8_t)(x.subface < 0 ? sl : 0);
        t.nu = (int16_t)U;
        ab.rt_taylor_tiles.push_back(t);
      }
      continue;
    }
    for (int sl = 0; sl < nsub; ++sl)
      for (int64_t u0 = 0; u0 < U; u0 += 128)
        ab.rt_tiles.push_back({(int32_t)it, (int16_t)sl, (int16_t)ab.item_class[it], (int16_t)u0,
                               (int16_t)std::min<int64_t>(128, U - u0)});
  }
  return ab;
}

}  // namespace amr

// ---------------------------------------------------------------------------
// Forward sparse rows for the CSR kernels.
// ---------------------------------------------------------------------------
namespace amr {

bool csr_routed(const amr_transfer_desc& desc, const amr_transfer_item&) {
  return (desc.flags & AMR_FLAG_CSR) != 0;
}

LsTables build_ls_tables(const amr_transfer_desc& desc) {
  LsTables lt;
  std::map<std::tuple<int, int, int>, int64_t> blocks;
  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    if (x.scheme != 1 || csr_routed(desc, x)) {
      lt.item_off.push_back(-1);
      continue;
    }
    const int p = x.patch_size, k = x.overlap, order = x.order;
    auto key = std::make_tuple(p, k, order);
    auto f = blocks.find(key);
    if (f == blocks.end()) {
      const int64_t off = (int64_t)lt.wd.size();
      lt.wd.resize(off + LS_BLOCK, 0.0);
      double* W = lt.wd.data() + off;
      double* sums = W + LS_CLASSES * LS_SLOTS * LS_NALPHA;
      const std::vector<std::array<int, 3>> alphas = taylor_alphas(order);
      for (int cls = 0; cls < LS_CLASSES; ++cls) {
        const int a = ls_class_rep(cls % 5, p), b = ls_class_rep(cls / 5, p);
        if (a < 0 || a >= p || b < 0 || b >= p) continue;
        const int c[3] = {-1, a, b}, lo[3] = {-k, 0, 0}, hi[3] = {k - 1, p - 1, p - 1};
        int ps[3], pl[3], ms[3], ml[3];
        for (int d = 0; d < 3; ++d) {
          stencil_window(c[d], lo[d], hi[d], pure_exactness(order), ps[d], pl[d]);
          stencil_window(c[d], lo[d], hi[d], mixed_exactness(order), ms[d], ml[d]);
        }
        // the kernel's slots and their points
        std::vector<std::pair<int, std::array<int, 3>>> slots;
        for (int d = 0; d < 3; ++d)
          for (int i = 0; i < pl[d]; ++i) {
            std::array<int, 3> xq{c[0], c[1], c[2]};
            xq[d] = ps[d] + i;
            slots.push_back({d * 5 + i, xq});
          }
        for (int q = 0; q < 3; ++q)
          for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i)
              slots.push_back({15 + (q * 3 + j) * 3 + i, {ms[0] + i, ms[1] + j, ms[2] + q}});
        // each support point (but the centre) on its first slot
        std::set<std::array<int, 3>> support;
        for (auto& xq : stencil_support(c, lo, hi, order))
          if (xq[0] != c[0] || xq[1] != c[1] || xq[2] != c[2]) support.insert(xq);
        std::vector<int> slot_of;
        std::vector<std::array<int, 3>> rel;
        std::set<std::array<int, 3>> done;
        for (auto& [sl, xq] : slots)
          if (support.count(xq) && !done.count(xq)) {
            done.insert(xq);
            slot_of.push_back(sl);
            rel.push_back({xq[0] - c[0], xq[1] - c[1], xq[2] - c[2]});
          }
        if (done.size() != support.size()) std::abort();  // the slots cover the support by construction
        const std::vector<std::vector<long double>> coef = ls_fit(rel, order);
        for (size_t al = 0; al < alphas.size(); ++al) {
          long double scale = 1;
          for (int d = 0; d < 3; ++d) scale *= factorial(alphas[al][d]) * std::pow(3.0L, alphas[al][d]);
          long double sum = 0;
          for (size_t q = 0; q < rel.size(); ++q) {
            const long double w = coef[al][q] / scale;
            W[(cls * LS_SLOTS + slot_of[q]) * LS_NALPHA + al] = (double)w;
            sum += w;
          }
          sums[cls * LS_NALPHA + al] = (double)sum;
        }
      }
      f = blocks.emplace(key, off).first;
    }
    lt.item_off.push_back(f->second);
  }
  lt.wf.assign(lt.wd.begin(), lt.wd.end());
  return lt;
}

CsrBuild build_csr(const amr_transfer_desc& desc) {
  CsrBuild cb;
  cb.pf.row_ptr.push_back(0);
  cb.rf.row_ptr.push_back(0);
  struct ClassRows { int32_t p0, np, r0, nr; };
  std::map<std::tuple<int, int, int, int>, ClassRows> classes;
  auto append = [](CsrFwd& f, const Rows& rows, auto base_of) {
    for (size_t i = 0; i < rows.rows.size(); ++i) {
      for (auto& [c, w] : rows.rows[i]) {
        f.col.push_back(c);
        f.val.push_back(w);
      }
      f.row_ptr.push_back((int32_t)f.col.size());
      f.out_vol.push_back(rows.out_vol[i]);
      f.base_vol.push_back(base_of(rows.out_vol[i]));
    }
  };
  for (int64_t it = 0; it < desc.num_items; ++it) {
    const amr_transfer_item& x = desc.items[it];
    cb.routed.push_back(csr_routed(desc, x) ? 1 : 0);
    if (!cb.routed.back()) continue;
    const int p = x.patch_size, k = x.overlap, m = x.order;
    auto key = std::make_tuple(p, k, m * 2 + x.scheme, x.subface);
    auto f = classes.find(key);
    if (f == classes.end()) {
      ClassRows cr{(int32_t)cb.pf.out_vol.size(), 0, (int32_t)cb.rf.out_vol.size(), 0};
      const int nsub = x.subface < 0 ? 9 : 1;
      for (int sl = 0; sl < nsub; ++sl) {
        const int sub = x.subface < 0 ? sl : x.subface;
        const int s0 = sub % 3, s1 = sub / 3;
        // interpolation: the base is the coarse centre (layer -1) nearest to the fine volume
        append(cb.pf, interpolation_rows(sub, sl, p, k, m, x.scheme), [&](uint32_t v) {
          const int q1 = (int)((v >> 6) & 63u), q0 = (int)(v & 63u);
          return pack_vol(0, k - 1, (s1 * p + q1) / 3, (s0 * p + q0) / 3);
        });
        // restriction: the base is the fine cell the expansion is about
        append(cb.rf, restriction_rows(sub, sl, p, k, m, x.scheme), [&](uint32_t v) {
          const int lk = (int)((v >> 12) & 7u), b = (int)((v >> 6) & 63u), a = (int)(v & 63u);
          const int j = lk - k;
          const int i = m == AMR_ORDER_DLINEAR ? 0 : std::min(3 * j + 1, k - 1);
          return pack_vol(sl, i + k, 3 * b + 1 - s1 * p, 3 * a + 1 - s0 * p);
        });
      }
      cr.np = (int32_t)cb.pf.out_vol.size() - cr.p0;
      cr.nr = (int32_t)cb.rf.out_vol.size() - cr.r0;
      f = classes.emplace(key, cr).first;
    }
    const ClassRows& cr = f->second;
    const int RT = 32;  // rows per tile
    for (int r = 0; r < cr.np; r += RT)
      cb.ptiles.push_back({(int32_t)it, cr.p0 + r, std::min(RT, cr.np - r), 0, 0});
    for (int r = 0; r < cr.nr; r += RT)
      cb.rtiles.push_back({(int32_t)it, cr.r0 + r, std::min(RT, cr.nr - r), 0, 0});
  }
  cb.p_nnz = (int64_t)cb.pf.col.size();
  cb.r_nnz = (int64_t)cb.rf.col.size();
  return cb;
}

}  // namespace amr
