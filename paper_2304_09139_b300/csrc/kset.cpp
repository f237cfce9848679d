// kset.cpp -- wavevector set, internal column order, table layout and tile plans (host C++).
#include "kset.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

namespace ssh {

int64_t chi_to_m(int d, int64_t N, double chi) {
  double x = chi * (double)d * (double)(N - 1);
  return (int64_t)std::nearbyint(x);  // round to nearest, ties to even (default rounding mode)
}

namespace {

struct Vec {
  int64_t n2;  // the norm that orders the set: |n|^2, or sum_a c_a n_a^2 for an anisotropic region
  int32_t c[kMaxDim];
};

bool half_space(const int32_t* c, int d) {
  for (int a = 0; a < d; a++) {
    if (c[a] != 0) return c[a] > 0;
  }
  return false;
}

// All n in H with sum_a w_a n_a^2 <= r2 (w_a >= 1 integers; all 1: the ball |n|^2 <= r2), visited axis by axis
// (odometer over the box |n_a| <= R_a, R_a = floor(sqrt(r2 / w_a))).
void collect(int d, const int64_t* w, int64_t r2, std::vector<Vec>* out) {
  int64_t R[kMaxDim] = {0, 0, 0, 0};
  for (int a = 0; a < d; a++) {
    int64_t r = (int64_t)std::floor(std::sqrt((double)r2 / (double)w[a]));
    while (w[a] * (r + 1) * (r + 1) <= r2) r++;
    while (r > 0 && w[a] * r * r > r2) r--;
    R[a] = r;
  }
  int32_t c[kMaxDim] = {0, 0, 0, 0};
  for (int a = 0; a < d; a++) c[a] = (int32_t)-R[a];
  out->clear();
  for (;;) {
    int64_t s = 0;
    for (int a = 0; a < d; a++) s += w[a] * (int64_t)c[a] * c[a];
    if (s <= r2 && half_space(c, d)) {
      Vec v;
      v.n2 = s;
      for (int a = 0; a < kMaxDim; a++) v.c[a] = a < d ? c[a] : 0;
      out->push_back(v);
    }
    int a = d - 1;
    while (a >= 0 && c[a] == R[a]) { c[a] = (int32_t)-R[a]; a--; }
    if (a < 0) break;
    c[a]++;
  }
}

bool pub_less(const Vec& x, const Vec& y, int d) {
  if (x.n2 != y.n2) return x.n2 < y.n2;
  for (int a = 0; a < d; a++)
    if (x.c[a] != y.c[a]) return x.c[a] < y.c[a];
  return false;
}

}  // namespace

// The set's public order is v's; internal order: prefix lexicographic, then last component.
static void fill_kset(int d, double L, const std::vector<Vec>& v, KSet* out) {
  const int64_t M = (int64_t)v.size();
  KSet& ks = *out;
  ks = KSet();
  ks.d = d;
  ks.M = M;
  ks.n_pub.resize((size_t)M * d);
  int64_t n2max = 0;
  for (int64_t i = 0; i < M; i++) {
    int64_t n2 = 0;
    for (int a = 0; a < d; a++) {
      ks.n_pub[i * d + a] = v[i].c[a];
      n2 += (int64_t)v[i].c[a] * v[i].c[a];
    }
    n2max = std::max(n2max, n2);
  }
  ks.k2max = (2.0 * M_PI / L) * (2.0 * M_PI / L) * (double)n2max;
  std::vector<int64_t> idx((size_t)M);
  for (int64_t i = 0; i < M; i++) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
    for (int a = 0; a < d; a++)
      if (v[x].c[a] != v[y].c[a]) return v[x].c[a] < v[y].c[a];
    return false;
  });
  ks.n_int.resize((size_t)M * d);
  ks.int2pub = idx;
  for (int a = 0; a < kMaxDim; a++) { ks.nmin[a] = 0; ks.nmax[a] = 0; }
  for (int64_t i = 0; i < M; i++) {
    for (int a = 0; a < d; a++) {
      int32_t c = v[idx[i]].c[a];
      ks.n_int[i * d + a] = c;
      if (i == 0 || c < ks.nmin[a]) ks.nmin[a] = c;
      if (i == 0 || c > ks.nmax[a]) ks.nmax[a] = c;
    }
  }
}

// The set of an exclusion region sum_a w_a n_a^2 <= R^2 (w = NULL: the ball), in the order (that norm, then
// lexicographic on the signed components).  K mode: every n in H with the norm <= (K L / 2 pi)^2 (1 + 1e-12);
// chi mode: the first M = round-half-even(chi d (N - 1)).
static int region_vectors(int d, int64_t N, double L, double chi, double K, const int32_t* wts, std::vector<Vec>* out) {
  if (d < 1 || d > kMaxDim || N < 1 || !(L > 0) || !std::isfinite(L)) return -1;
  if ((chi > 0) == (K > 0)) return -1;
  int64_t w[kMaxDim] = {1, 1, 1, 1};
  if (wts)
    for (int a = 0; a < d; a++) {
      if (wts[a] < 1 || wts[a] > 1 << 20) return -1;
      w[a] = wts[a];
    }
  std::vector<Vec>& v = *out;
  int64_t M;
  if (K > 0) {
    long double rr = (long double)K * (long double)L / (2.0L * 3.14159265358979323846264338327950288L);
    int64_t r2 = (int64_t)std::floor(rr * rr * (1.0L + 1e-12L));
    collect(d, w, r2, &v);
    M = (int64_t)v.size();
  } else {
    M = chi_to_m(d, N, chi);
    if (M < 0) return -1;
    // smallest region holding M half-space vectors: its volume V_d R^d / (2 sqrt(prod w)) ~ M, then grow
    double wprod = 1.0;
    for (int a = 0; a < d; a++) wprod *= (double)w[a];
    double est = std::pow(2.0 * (double)M + 1.0, 2.0 / d) * std::pow(wprod, 1.0 / d);
    int64_t r2 = std::max<int64_t>(1, (int64_t)est);
    for (;;) {
      collect(d, w, r2, &v);
      if ((int64_t)v.size() >= M) break;
      r2 = r2 + r2 / 4 + 1;
    }
  }
  std::sort(v.begin(), v.end(), [d](const Vec& x, const Vec& y) { return pub_less(x, y, d); });
  v.resize((size_t)M);
  return 0;
}

int build_kset(int d, int64_t N, double L, double chi, double K, KSet* out) {
  std::vector<Vec> v;
  if (region_vectors(d, N, L, chi, K, nullptr, &v) != 0) return -1;
  fill_kset(d, L, v, out);
  return 0;
}

int kset_region(int d, int64_t N, double L, double chi, double K, const int32_t* w, std::vector<int32_t>* n) {
  std::vector<Vec> v;
  if (region_vectors(d, N, L, chi, K, w, &v) != 0) return -1;
  n->resize(v.size() * d);
  for (size_t i = 0; i < v.size(); i++)
    for (int a = 0; a < d; a++) (*n)[i * d + a] = v[i].c[a];
  return 0;
}

int build_kset_list(int d, int64_t M, const int32_t* n, double L, KSet* out) {
  if (d < 1 || d > kMaxDim || M < 1 || !n || !(L > 0) || !std::isfinite(L)) return -1;
  std::vector<Vec> v((size_t)M);
  for (int64_t i = 0; i < M; i++) {
    Vec& x = v[i];
    x.n2 = 0;
    for (int a = 0; a < kMaxDim; a++) x.c[a] = a < d ? n[i * d + a] : 0;
    for (int a = 0; a < d; a++)
      if (x.c[a] < -32767 || x.c[a] > 32767) return -1;
    if (!half_space(x.c, d)) return -1;
  }
  std::vector<Vec> s = v;  // every vector once
  std::sort(s.begin(), s.end(), [d](const Vec& x, const Vec& y) { return pub_less(x, y, d); });
  for (size_t i = 1; i < s.size(); i++)
    if (!pub_less(s[i - 1], s[i], d)) return -1;
  fill_kset(d, L, v, out);
  return 0;
}

static int32_t floordiv(int32_t a, int32_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

TableLayout build_table_layout(const KSet& ks) {
  TableLayout tl;
  int d = ks.d;
  int32_t r = 0;
  for (int a = 0; a + 1 < d; a++) {
    tl.pre_base[a] = r;
    for (int32_t c = ks.nmin[a]; c <= ks.nmax[a]; c++) tl.rows.push_back({a, c}), r++;
  }
  if (ks.M > 0) {
    tl.qmin = floordiv(ks.nmin[d - 1], kDigit);
    tl.qmax = floordiv(ks.nmax[d - 1], kDigit);
  }
  tl.hi_base = r;
  for (int32_t q = tl.qmin; q <= tl.qmax; q++) tl.rows.push_back({d - 1, q * kDigit}), r++;
  tl.lo_base = r;
  for (int32_t q = 0; q < kDigit; q++) tl.rows.push_back({d - 1, q}), r++;
  return tl;
}

NtPlan build_nt_plan(const KSet& ks, const TableLayout& tl) {
  NtPlan p;
  int d = ks.d;
  // slots: runs of <= kSlotK vectors in one column and one high digit
  struct Raw { int64_t k0; int cnt; int32_t pre[kMaxDim]; int32_t q; int32_t r0; };
  std::vector<Raw> raw;
  int64_t i = 0;
  while (i < ks.M) {
    const int32_t* n = &ks.n_int[i * d];
    int32_t q = floordiv(n[d - 1], kDigit);
    Raw s;
    s.k0 = i;
    s.cnt = 1;
    for (int a = 0; a < kMaxDim; a++) s.pre[a] = a + 1 < d ? n[a] : 0;
    s.q = q;
    s.r0 = n[d - 1] - q * kDigit;
    int64_t j = i + 1;
    while (j < ks.M && s.cnt < kSlotK) {
      const int32_t* m = &ks.n_int[j * d];
      bool same = true;
      for (int a = 0; a + 1 < d; a++) same = same && m[a] == n[a];
      if (!same || m[d - 1] != n[d - 1] + s.cnt || floordiv(m[d - 1], kDigit) != q) break;
      s.cnt++;
      j++;
    }
    raw.push_back(s);
    i = j;
  }
  // blocks of kNtThreads slots; each block gets the list of distinct (prefix, q) it needs
  for (size_t b0 = 0; b0 < raw.size(); b0 += kNtThreads) {
    size_t b1 = std::min(raw.size(), b0 + kNtThreads);
    NtBlock blk;
    blk.slot0 = (int32_t)b0;
    blk.nslots = (int32_t)(b1 - b0);
    blk.g0 = (int32_t)(p.g_rows.size() / kMaxDim);
    std::map<std::tuple<int32_t, int32_t, int32_t, int32_t>, int> gmap;
    for (size_t s = b0; s < b1; s++) {
      const Raw& r = raw[s];
      auto key = std::make_tuple(r.pre[0], r.pre[1], r.pre[2], r.q);
      auto it = gmap.find(key);
      int g;
      if (it == gmap.end()) {
        g = (int)gmap.size();
        gmap[key] = g;
        for (int a = 0; a + 1 < d; a++) p.g_rows.push_back(tl.pre_base[a] + r.pre[a] - ks.nmin[a]);
        for (int a = d - 1; a + 1 < kMaxDim; a++) p.g_rows.push_back(-1);
        p.g_rows.push_back(tl.hi_base + r.q - tl.qmin);
      } else {
        g = it->second;
      }
      NtSlot sl;
      sl.k0 = (int32_t)r.k0;
      sl.cnt = (int16_t)r.cnt;
      sl.g = (int16_t)g;
      sl.r0 = (int16_t)r.r0;
      sl.pad[0] = sl.pad[1] = sl.pad[2] = 0;
      p.slots.push_back(sl);
    }
    blk.ng = (int32_t)gmap.size();
    p.max_ng = std::max(p.max_ng, blk.ng);
    p.blocks.push_back(blk);
  }
  return p;
}

FPlan build_f_plan(const KSet& ks, const TableLayout& tl) {
  FPlan p;
  int d = ks.d;
  int64_t i = 0;
  while (i < ks.M) {
    const int32_t* n = &ks.n_int[i * d];
    FCol c;
    c.k0 = (int32_t)i;
    c.nlo = n[d - 1];
    c.pad = 0;
    for (int a = 0; a + 1 < kMaxDim; a++) {
      c.pre[a] = a + 1 < d ? n[a] : 0;
      c.rows[a] = a + 1 < d ? tl.pre_base[a] + n[a] - ks.nmin[a] : -1;
    }
    int64_t j = i + 1;
    while (j < ks.M) {
      const int32_t* m = &ks.n_int[j * d];
      bool same = m[d - 1] == n[d - 1] + (int32_t)(j - i);  // a column is a contiguous run
      for (int a = 0; a + 1 < d; a++) same = same && m[a] == n[a];
      if (!same) break;
      j++;
    }
    c.len = (int32_t)(j - i);
    p.cols.push_back(c);
    i = j;
  }
  return p;
}

}  // namespace ssh
