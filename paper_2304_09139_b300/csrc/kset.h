// kset.h -- the independent wavevectors of the periodic box and the tile plans built on them (host C++).
//
// Definitions (arXiv:2304.09139): the box has side L, so k = 2 pi n / L with n integer; S(k) = S(-k), so of
// the 2M+1 lattice vectors with |k| <= K (counting k = 0) only M are independent, and chi = M / (d (N-1)).
// The library keeps the half-space H = {n != 0 : first non-zero component > 0}.
//   K mode   : every n in H with |n|^2 <= (K L / 2 pi)^2 (1 + 1e-12)      (complete shells)
//   chi mode : the M = round-half-even(chi d (N-1)) first vectors of H in the order (|n|^2, lexicographic)
// Public order: (|n|^2, then lexicographic on the signed components).
// Internal order: "columns" -- vectors grouped by their first d-1 components (the prefix, lexicographic),
// the last component ascending.  In either mode a column is a contiguous run of the last component.
#pragma once
#include <stdint.h>

#include <vector>

namespace ssh {

constexpr int kMaxDim = 4;
constexpr int kDigit = 32;  // the last axis is split as n_d = q * kDigit + r, 0 <= r < kDigit

struct KSet {
  int d = 0;
  int64_t M = 0;
  std::vector<int32_t> n_pub;    // [M][d] public order
  std::vector<int32_t> n_int;    // [M][d] internal (column) order
  std::vector<int64_t> int2pub;  // internal index -> public index
  int32_t nmin[kMaxDim] = {0, 0, 0, 0}, nmax[kMaxDim] = {0, 0, 0, 0};
  double k2max = 0;              // max |k|^2 = (2 pi / L)^2 max |n|^2
};

// Returns 0 on success, -1 on bad arguments.
int build_kset(int d, int64_t N, double L, double chi, double K, KSet* out);
// An anisotropic exclusion region sum_a w_a n_a^2 <= R^2 (integer w_a >= 1), in either mode, as a list in the
// order (that norm, lexicographic): the vectors only.
int kset_region(int d, int64_t N, double L, double chi, double K, const int32_t* w, std::vector<int32_t>* n);
// A given list of distinct half-space vectors (|n_a| <= 32767); the public order is the list's.
int build_kset_list(int d, int64_t M, const int32_t* n, double L, KSet* out);
int64_t chi_to_m(int d, int64_t N, double chi);

// ---- per-particle power tables: row r holds e^{2 pi i m s_{j,axis}} for every particle j
struct TabRow {
  int32_t axis;
  int32_t m;
};

struct TableLayout {
  std::vector<TabRow> rows;
  int32_t pre_base[kMaxDim] = {0, 0, 0, 0};  // row of prefix axis a, component value v: pre_base[a] + v - nmin[a]
  int32_t hi_base = 0, qmin = 0, qmax = -1;  // row of last-axis high digit q: hi_base + q - qmin
  int32_t lo_base = 0;                       // row of last-axis low digit r: lo_base + r
};

TableLayout build_table_layout(const KSet& ks);

// ---- collective density plan (thread <-> up to kSlotK consecutive vectors of one column and one digit)
constexpr int kSlotK = 4;
constexpr int kNtThreads = 256;

struct NtSlot {   // 16 bytes
  int32_t k0;     // internal index of the first vector
  int16_t cnt;    // 1..kSlotK
  int16_t g;      // local index of the (prefix, q) product row in the block's G list
  int16_t r0;     // low digit of the first vector
  int16_t pad[3];
};

struct NtBlock {
  int32_t slot0, nslots;
  int32_t g0, ng;  // G list entries [g0, g0+ng) of the plan's gl_rows
};

struct NtPlan {
  std::vector<NtSlot> slots;
  std::vector<NtBlock> blocks;
  std::vector<int32_t> g_rows;  // per G entry: kMaxDim global rows (prefix axes 0..d-2, then the q row), -1 unused
  int max_ng = 0;
};

NtPlan build_nt_plan(const KSet& ks, const TableLayout& tl);

// ---- force plan (thread <-> particle, walking columns)
struct FCol {        // 32 bytes
  int32_t k0, len, nlo;
  int32_t rows[kMaxDim - 1];  // global rows of the prefix components
  int32_t pre[kMaxDim - 1];   // prefix component values
  int32_t pad;
};

struct FPlan {
  std::vector<FCol> cols;
};

FPlan build_f_plan(const KSet& ks, const TableLayout& tl);

}  // namespace ssh
