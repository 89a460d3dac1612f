// Host-side set-up of the nle library: CSR validation, the IC(lfil, tau_IC)
// factor (Section 2), the level sets of L and L^T, the optional multicolour
// ordering, the slab-major level-minor relabelling and the packing of the
// sliced-ELL and per-slab ELL matrices.
//
// The factor is the preconditioner Phat_0 = (L L^T)^{-1} of Section 2.  The
// paper does not print the IC variant; the library uses a left-looking column
// algorithm whose every floating-point operation happens in a fixed order
// (stated in include/nle.h), so that its drop decisions are reproducible.
// Implementation: columns of L are kept in compressed form; a "next entry"
// cursor per finished column k points at its first row >= the column being
// built, and per-row buckets list the columns whose cursor sits on that row
// (so column j finds every k with L(j,k) != 0 without scanning).
#include "nle_setup.h"

#include "nle_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace nle {

int validate_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci, const double *va, std::string &msg) {
  if (rp[0] != 0 || rp[n] != nnz) {
    msg = "rowptr[0] must be 0 and rowptr[n] must equal nnz";
    return 2;
  }
  std::vector<int64_t> cnt(n + 1, 0);
  for (int64_t i = 0; i < n; i++) {
    if (rp[i + 1] < rp[i]) {
      msg = "rowptr is not monotone";
      return 2;
    }
    bool diag = false;
    for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
      const int64_t c = ci[e];
      if (c < 0 || c >= n) {
        msg = "column index out of range in row " + std::to_string(i);
        return 2;
      }
      if (e > rp[i] && ci[e - 1] >= c) {
        msg = "columns not strictly ascending in row " + std::to_string(i);
        return 2;
      }
      if (c == i) {
        diag = true;
        if (!(va[e] > 0.0)) {
          msg = "non-positive diagonal in row " + std::to_string(i);
          return 3;
        }
      }
      if (!std::isfinite(va[e])) {
        msg = "non-finite value in row " + std::to_string(i);
        return 2;
      }
      cnt[c + 1]++;
    }
    if (!diag) {
      msg = "missing diagonal in row " + std::to_string(i);
      return 2;
    }
  }
  // symmetry: build the transpose and compare entry by entry
  for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  std::vector<int32_t> tc(nnz);
  std::vector<double> tv(nnz);
  for (int64_t i = 0; i < n; i++)
    for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
      const int64_t c = ci[e];
      tc[fill[c]] = (int32_t)i;
      tv[fill[c]] = va[e];
      fill[c]++;
    }
  for (int64_t i = 0; i < n; i++) {
    if (cnt[i + 1] - cnt[i] != rp[i + 1] - rp[i]) {
      msg = "pattern is not symmetric (row " + std::to_string(i) + ")";
      return 2;
    }
    for (int64_t e = rp[i], f = cnt[i]; e < rp[i + 1]; e++, f++) {
      if (tc[f] != ci[e]) {
        msg = "pattern is not symmetric (row " + std::to_string(i) + ")";
        return 2;
      }
      const double a = va[e], b = tv[f];
      if (std::fabs(a - b) > 1e-12 * std::max(std::fabs(a), std::fabs(b))) {
        msg = "values are not symmetric (row " + std::to_string(i) + ")";
        return 2;
      }
    }
  }
  return 0;
}

int ic_factor_host(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, int lfil, double tau,
                   Factor &F, int64_t *bad_col) {
  // columns of L: colstart (n+1), rows / values appended column by column
  std::vector<int64_t> cs(n + 1, 0);
  std::vector<int32_t> rows;
  std::vector<double> vals;
  rows.reserve((size_t)n * (size_t)(std::min<int64_t>(lfil, n) + 1));
  vals.reserve(rows.capacity());
  std::vector<int64_t> cursor(n, -1);   // next entry of column k to apply
  std::vector<int64_t> bhead(n, -1);    // bucket of row i: columns whose cursor row is i
  std::vector<int64_t> bnext(n, -1);
  std::vector<double> w(n, 0.0);
  std::vector<int64_t> mark(n, -1);
  std::vector<int64_t> touched;
  std::vector<int64_t> ks;
  struct Cand {
    int64_t i;
    double v, a;
  };
  std::vector<Cand> cand;
  auto push_bucket = [&](int64_t k) {
    const int64_t r = rows[cursor[k]];
    bnext[k] = bhead[r];
    bhead[r] = k;
  };
  for (int64_t j = 0; j < n; j++) {
    touched.clear();
    // column j of A from row j (symmetric storage), and ||A(:,j)||_2 summed
    // over the whole row in ascending column order
    double nrm2 = 0.0;
    for (int64_t e = rp[j]; e < rp[j + 1]; e++) {
      const double a = va[e];
      nrm2 += a * a;
      const int64_t i = ci[e];
      if (i >= j) {
        if (mark[i] != j) {
          mark[i] = j;
          touched.push_back(i);
          w[i] = 0.0;
        }
        w[i] += a;
      }
    }
    const double anorm = std::sqrt(nrm2);
    // columns k < j with L(j,k) != 0, in ascending k
    ks.clear();
    for (int64_t k = bhead[j]; k >= 0; k = bnext[k]) ks.push_back(k);
    bhead[j] = -1;
    std::sort(ks.begin(), ks.end());
    for (int64_t k : ks) {
      const int64_t e0 = cursor[k];
      const double ljk = vals[e0];
      for (int64_t e = e0; e < cs[k + 1]; e++) {
        const int64_t i = rows[e];
        if (mark[i] != j) {
          mark[i] = j;
          touched.push_back(i);
          w[i] = 0.0;
        }
        w[i] -= vals[e] * ljk;
      }
      cursor[k] = e0 + 1;
      if (cursor[k] < cs[k + 1]) push_bucket(k);
    }
    const double d = w[j];
    if (!(d > 0.0)) {
      if (bad_col) *bad_col = j;
      return -2;
    }
    const double ljj = std::sqrt(d);
    cand.clear();
    for (int64_t i : touched) {
      if (i == j) continue;
      const double lij = w[i] / ljj;
      if (!(std::fabs(lij) < tau * anorm)) cand.push_back({i, lij, std::fabs(lij)});
    }
    if ((int64_t)cand.size() > lfil) {
      auto bigger = [](const Cand &x, const Cand &y) { return x.a > y.a || (x.a == y.a && x.i < y.i); };
      std::nth_element(cand.begin(), cand.begin() + lfil, cand.end(), bigger);
      cand.resize(lfil);
    }
    std::sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.i < y.i; });
    rows.push_back((int32_t)j);
    vals.push_back(ljj);
    for (const Cand &c : cand) {
      rows.push_back((int32_t)c.i);
      vals.push_back(c.v);
    }
    cs[j + 1] = (int64_t)rows.size();
    if (!cand.empty()) {
      cursor[j] = cs[j] + 1;
      push_bucket(j);
    }
  }
  factor_from_columns(n, std::move(cs), std::move(rows), std::move(vals), F);
  return 0;
}

void factor_from_columns(int64_t n, std::vector<int64_t> cs, std::vector<int32_t> rows, std::vector<double> vals,
                         Factor &F) {
  // L by rows (diagonal last), from the columns
  const int64_t nnz = (int64_t)rows.size();
  F.n = n;
  F.Lrowptr.assign(n + 1, 0);
  for (int64_t e = 0; e < nnz; e++) F.Lrowptr[rows[e] + 1]++;
  for (int64_t i = 0; i < n; i++) F.Lrowptr[i + 1] += F.Lrowptr[i];
  F.Lcol.resize(nnz);
  F.Lval.resize(nnz);
  std::vector<int64_t> fill(F.Lrowptr.begin(), F.Lrowptr.end() - 1);
  for (int64_t k = 0; k < n; k++)
    for (int64_t e = cs[k]; e < cs[k + 1]; e++) {
      const int64_t i = rows[e];
      F.Lcol[fill[i]] = (int32_t)k;
      F.Lval[fill[i]] = vals[e];
      fill[i]++;
    }
  F.Ccolptr = std::move(cs);
  F.Crow = std::move(rows);
  F.Cval = std::move(vals);
  // levels: L by pushing along columns (ascending), U = L^T by pulling
  // along columns (descending)
  F.levL.assign(n, 0);
  F.levU.assign(n, 0);
  for (int64_t k = 0; k < n; k++)
    for (int64_t e = F.Ccolptr[k] + 1; e < F.Ccolptr[k + 1]; e++) {
      const int64_t i = F.Crow[e];
      F.levL[i] = std::max(F.levL[i], F.levL[k] + 1);
    }
  for (int64_t k = n - 1; k >= 0; k--) {
    int32_t l = 0;
    for (int64_t e = F.Ccolptr[k] + 1; e < F.Ccolptr[k + 1]; e++) l = std::max(l, F.levU[F.Crow[e]] + 1);
    F.levU[k] = l;
  }
  F.nlevL = 0;
  F.nlevU = 0;
  for (int64_t i = 0; i < n; i++) {
    F.nlevL = std::max<int64_t>(F.nlevL, F.levL[i] + 1);
    F.nlevU = std::max<int64_t>(F.nlevU, F.levU[i] + 1);
  }
}

// Greedy colouring in natural order: row i takes the smallest colour not
// held by an already coloured row of its neighbourhood ({j != i : A_ij != 0},
// plus the neighbours of those rows for distance 2).  used[c] == i + 1
// marks colour c as taken for row i, so the marks need no clearing.
int32_t multicolor_order(int64_t n, const int64_t *rp, const int32_t *ci, int distance, std::vector<int32_t> &perm) {
  std::vector<int32_t> color(n, -1);
  std::vector<int64_t> used;
  int32_t ncol = 0;
  for (int64_t i = 0; i < n; i++) {
    auto take = [&](int64_t j) {
      if (j == i || color[j] < 0) return;
      const int32_t c = color[j];
      if ((size_t)c >= used.size()) used.resize((size_t)c + 1, 0);
      used[c] = i + 1;
    };
    for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
      const int64_t j = ci[e];
      take(j);
      if (distance == 2)
        for (int64_t f = rp[j]; f < rp[j + 1]; f++) take(ci[f]);
    }
    int32_t c = 0;
    while ((size_t)c < used.size() && used[c] == i + 1) c++;
    color[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  // counting sort by colour, stable in the row index
  std::vector<int64_t> start((size_t)ncol + 1, 0);
  for (int64_t i = 0; i < n; i++) start[color[i] + 1]++;
  for (int32_t c = 0; c < ncol; c++) start[c + 1] += start[c];
  perm.assign(n, 0);
  for (int64_t i = 0; i < n; i++) perm[start[color[i]]++] = (int32_t)i;
  return ncol;
}

void permute_csr(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, const std::vector<int32_t> &perm,
                 std::vector<int64_t> &brp, std::vector<int32_t> &bci, std::vector<double> &bva) {
  std::vector<int32_t> iperm(n);
  for (int64_t k = 0; k < n; k++) iperm[perm[k]] = (int32_t)k;
  brp.assign(n + 1, 0);
  for (int64_t k = 0; k < n; k++) brp[k + 1] = brp[k] + (rp[perm[k] + 1] - rp[perm[k]]);
  bci.resize(brp[n]);
  bva.resize(brp[n]);
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t k = 0; k < n; k++) {
    const int64_t i = perm[k];
    row.clear();
    for (int64_t e = rp[i]; e < rp[i + 1]; e++) row.emplace_back(iperm[ci[e]], va[e]);
    std::sort(row.begin(), row.end(), [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
      return a.first < b.first;
    });
    for (size_t t = 0; t < row.size(); t++) {
      bci[brp[k] + (int64_t)t] = row[t].first;
      bva[brp[k] + (int64_t)t] = row[t].second;
    }
  }
}

void slab_level_order(const Factor &F, int64_t bsize, const int32_t *locality, std::vector<int32_t> &perm,
                      std::vector<int32_t> &iperm) {
  const int64_t n = F.n;
  perm.resize(n);
  for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
  auto loc = [&](int32_t r) -> int64_t { return locality ? locality[r] : r; };
  // every slab holds bsize consecutive locality values, so sorting by
  // (slab, level, locality) fills each slab's position range exactly
  std::sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
    const int64_t sa = loc(a) / bsize, sb = loc(b) / bsize;
    if (sa != sb) return sa < sb;
    if (F.levL[a] != F.levL[b]) return F.levL[a] < F.levL[b];
    return loc(a) < loc(b);
  });
  iperm.assign(n, 0);
  for (int64_t p = 0; p < n; p++) iperm[perm[p]] = (int32_t)p;
}

// Pack rows of a matrix given row by row (in new numbering) into SELL.
template <typename TV>
static void pack(int64_t n, int64_t npad, int H, const std::vector<int64_t> &rp, const std::vector<int32_t> &col,
                 const std::vector<double> &val, int pad_mode, int64_t pad_col, SellHost<TV> &out) {
  const int64_t ns = npad / H;
  out.nslices = ns;
  out.sptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; s++) {
    int64_t w = 0;
    for (int64_t r = s * H; r < std::min(n, (s + 1) * H); r++) w = std::max(w, rp[r + 1] - rp[r]);
    out.sptr[s + 1] = out.sptr[s] + w * H;
  }
  out.col.assign(out.sptr[ns], 0);
  out.val.assign(out.sptr[ns], TV(0));
  for (int64_t s = 0; s < ns; s++) {
    const int64_t base = out.sptr[s];
    const int64_t w = (out.sptr[s + 1] - base) / H;
    for (int64_t q = 0; q < H; q++) {
      const int64_t r = s * H + q;
      const int64_t len = (r < n) ? rp[r + 1] - rp[r] : 0;
      for (int64_t e = 0; e < w; e++) {
        const int64_t idx = base + e * H + q;
        if (e < len) {
          out.col[idx] = col[rp[r] + e];
          out.val[idx] = TV(val[rp[r] + e]);
        } else {
          out.col[idx] = (int32_t)(pad_mode == 0 ? r : pad_col);
          out.val[idx] = TV(0);
        }
      }
    }
  }
}

// Per-slab ELL of a strictly triangular matrix given by rows (relabelled
// order), plus the round of every row inside its group of R rows (low
// nibble; the group's last round in the high nibble): the length
// of the longest dependency chain ending at the row within the group
// (lower: earlier rows of the group; upper: later rows).
template <typename TV>
static void ell(int64_t n, int64_t npad, int64_t bsize, bool lower, const std::vector<int64_t> &rp,
                const std::vector<int32_t> &col, const std::vector<double> &val, const std::vector<int32_t> *lev,
                int R, EllHost<TV> &out) {
  const int64_t ns = (npad + bsize - 1) / bsize;
  out.off.assign(ns + 1, 0);
  out.width.assign(ns, 8);
  for (int64_t s = 0; s < ns; s++) {
    int64_t w = 0;
    for (int64_t r = s * bsize; r < std::min(n, (s + 1) * bsize); r++) w = std::max(w, rp[r + 1] - rp[r]);
    w = std::max<int64_t>(8, (w + 7) / 8 * 8);
    out.width[s] = (int32_t)w;
    const int64_t rows = std::min(npad, (s + 1) * bsize) - s * bsize;
    out.off[s + 1] = out.off[s] + rows * w;
  }
  out.col.assign(out.off[ns], -1);
  out.val.assign(out.off[ns], TV(0));
  for (int64_t s = 0; s < ns; s++)
    for (int64_t r = s * bsize; r < std::min(n, (s + 1) * bsize); r++) {
      const int64_t base = out.off[s] + (r - s * bsize) * out.width[s];
      for (int64_t e = rp[r]; e < rp[r + 1]; e++) {
        out.col[base + (e - rp[r])] = col[e];
        out.val[base + (e - rp[r])] = TV(val[e]);
      }
    }
  out.round.assign(npad, 0);
  for (int64_t g0 = 0; g0 < n; g0 += R) {
    const int64_t g1 = std::min(n, g0 + R);
    if (lev) {
      // one level per round: rank of the row's level among the group's
      // levels, ascending for L, descending for L^T
      for (int64_t r = g0; r < g1; r++) {
        int rank = 0;
        for (int64_t t = g0; t < g1; t++) {
          bool below = lower ? (*lev)[t] < (*lev)[r] : (*lev)[t] > (*lev)[r];
          for (int64_t u = g0; u < t && below; u++)
            if ((*lev)[u] == (*lev)[t]) below = false;  // count each level once
          rank += below;
        }
        out.round[r] = (uint16_t)rank;
      }
    } else if (lower) {
      for (int64_t r = g0; r < g1; r++)
        for (int64_t e = rp[r]; e < rp[r + 1]; e++)
          if (col[e] >= g0) out.round[r] = std::max<uint16_t>(out.round[r], out.round[col[e]] + 1);
    } else {
      for (int64_t r = g1 - 1; r >= g0; r--)
        for (int64_t e = rp[r]; e < rp[r + 1]; e++)
          if (col[e] < g1) out.round[r] = std::max<uint16_t>(out.round[r], out.round[col[e]] + 1);
    }
    // every row also carries the number of rounds of its group, less one,
    // in the high nibble (rounds <= R <= 4), so a warp needs no reduction
    // to learn it
    // (padding rows past n included: every lane of the group must agree)
    // and the group's overflow steps in the high byte: the entries of its
    // longest row past the TRSV_EPL * 32 / R prefetched ones, in steps of 32 / R,
    // so that the solve stops at the group's last entry, not the slab's width
    uint16_t last = 0;
    int64_t glen = 0;
    for (int64_t r = g0; r < g1; r++) {
      last = std::max(last, out.round[r]);
      glen = std::max<int64_t>(glen, rp[r + 1] - rp[r]);
    }
    const int64_t lanes = 32 / R, pre = TRSV_EPL * lanes;
    const int64_t steps = std::min<int64_t>(255, glen > pre ? (glen - pre + lanes - 1) / lanes : 0);
    for (int64_t r = g0; r < std::min(npad, g0 + R); r++)
      out.round[r] = (uint16_t)(out.round[r] | (last << 4) | (steps << 8));
  }
}

template <typename TV>
void build_sell(const Permuted &P, int H, int64_t bsize, bool level_rounds, int R, SellSet<TV> &S) {
  pack<TV>(P.n, P.npad, H, P.Arp, P.Acol, P.Aval, 0, 0, S.A);
  pack<double>(P.n, P.npad, H, P.Arp, P.Acol, P.Aval, 0, 0, S.A64);
  const std::vector<int32_t> *lev = level_rounds ? &P.lev : nullptr;
  ell<TV>(P.n, P.npad, bsize, true, P.Lrp, P.Lcol, P.Lval, lev, R, S.L);
  ell<TV>(P.n, P.npad, bsize, false, P.Urp, P.Ucol, P.Uval, lev, R, S.U);
  S.diag.assign(P.npad, TV(1));
  for (int64_t i = 0; i < P.n; i++) S.diag[i] = TV(1.0 / P.diag[i]);  // reciprocal pivots
}

template void build_sell<float>(const Permuted &, int, int64_t, bool, int, SellSet<float> &);
template void build_sell<double>(const Permuted &, int, int64_t, bool, int, SellSet<double> &);

template <typename TV>
void build_chain(const Permuted &P, int64_t bsize, bool lower, int nwarps, ChainHost<TV> &out) {
  const int64_t n = P.n, npad = P.npad;
  const std::vector<int64_t> &rp = lower ? P.Lrp : P.Urp;
  const std::vector<int32_t> &col = lower ? P.Lcol : P.Ucol;
  const std::vector<double> &val = lower ? P.Lval : P.Uval;
  const std::vector<int32_t> &lev = lower ? P.lev : P.levU;
  const int64_t ns = (npad + bsize - 1) / bsize;
  EllHost<TV> &E = out.ell;
  E.off.assign(ns + 1, 0);
  E.width.assign(ns, 8);
  for (int64_t s = 0; s < ns; s++) {
    int64_t w = 0;
    for (int64_t r = s * bsize; r < std::min(n, (s + 1) * bsize); r++) w = std::max(w, rp[r + 1] - rp[r]);
    w = std::max<int64_t>(8, (w + 7) / 8 * 8);
    E.width[s] = (int32_t)w;
    E.off[s + 1] = E.off[s] + (std::min(npad, (s + 1) * bsize) - s * bsize) * w;
  }
  E.col.assign(E.off[ns], -1);
  E.val.assign(E.off[ns], TV(0));
  E.round.clear();
  out.wptr.assign(ns * (NWARP + 1), 0);
  out.task.clear();
  out.nstrands = 0;
  // does row r depend on row q?  (columns ascending within a row)
  auto dep = [&](int64_t r, int64_t q) {
    if (r >= n || q < 0 || q >= n) return false;
    return std::binary_search(col.begin() + rp[r], col.begin() + rp[r + 1], (int32_t)q);
  };
  std::vector<int64_t> tfirst;  // per task of the slab: processing index of its first row
  std::vector<int> tcnt;
  std::vector<int64_t> sfirst;  // per strand: first task
  std::vector<int64_t> strand_of_row;
  for (int64_t s = 0; s < ns; s++) {
    const int64_t b0 = s * bsize, b1 = std::min(npad, b0 + bsize), nb = b1 - b0;
    if (nb <= 0) continue;
    auto row = [&](int64_t i) { return lower ? b0 + i : b1 - 1 - i; };
    // tasks: a row that depends on its predecessor continues the current
    // task; one that does not closes a task that holds such a link (a chain),
    // while rows without links are packed TRSV_ROWS to a task
    tfirst.clear();
    tcnt.clear();
    std::vector<char> tlinked;  // first row depends on the previous task's last row
    for (int64_t i = 0; i < nb;) {
      const bool linked = i > 0 && dep(row(i), row(i - 1));
      bool chainlike = linked;
      int cnt = 1;
      tfirst.push_back(i);
      tlinked.push_back(linked ? 1 : 0);
      i++;
      while (cnt < TRSV_ROWS && i < nb) {
        const bool l = dep(row(i), row(i - 1));
        if (!l && chainlike) break;
        chainlike = chainlike || l;
        cnt++;
        i++;
      }
      tcnt.push_back(cnt);
    }
    const int64_t nt = (int64_t)tfirst.size();
    // strands: runs of linked tasks
    sfirst.clear();
    for (int64_t t = 0; t < nt; t++)
      if (!tlinked[t]) sfirst.push_back(t);
    const int64_t nstr = (int64_t)sfirst.size();
    sfirst.push_back(nt);
    strand_of_row.assign(nb, 0);
    for (int64_t k = 0; k < nstr; k++)
      for (int64_t i = tfirst[sfirst[k]]; i < (sfirst[k + 1] < nt ? tfirst[sfirst[k + 1]] : nb); i++)
        strand_of_row[i] = k;
    // strand graph inside the slab and a topological order (Kahn) that takes
    // the ready strand whose first row has the lowest level first
    std::vector<std::vector<int64_t>> succ(nstr);
    std::vector<int64_t> indeg(nstr, 0), deps;
    for (int64_t k = 0; k < nstr; k++) {
      deps.clear();
      const int64_t i0 = tfirst[sfirst[k]], i1 = sfirst[k + 1] < nt ? tfirst[sfirst[k + 1]] : nb;
      for (int64_t i = i0; i < i1; i++) {
        const int64_t r = row(i);
        if (r >= n) continue;
        for (int64_t e = rp[r]; e < rp[r + 1]; e++) {
          const int64_t c = col[e];
          if (c < b0 || c >= b1) continue;
          const int64_t ci = lower ? c - b0 : b1 - 1 - c;
          const int64_t d = strand_of_row[ci];
          if (d != k) deps.push_back(d);
        }
      }
      std::sort(deps.begin(), deps.end());
      deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
      for (int64_t d : deps) {
        succ[d].push_back(k);
        indeg[k]++;
      }
    }
    auto key = [&](int64_t k) {
      const int64_t r = row(tfirst[sfirst[k]]);
      return std::make_pair(r < n ? (int64_t)lev[r] : (int64_t)0, tfirst[sfirst[k]]);
    };
    auto later = [&](int64_t a, int64_t b) { return key(a) > key(b); };
    std::vector<int64_t> heap, order;
    for (int64_t k = 0; k < nstr; k++)
      if (!indeg[k]) heap.push_back(k);
    std::make_heap(heap.begin(), heap.end(), later);
    while (!heap.empty()) {
      std::pop_heap(heap.begin(), heap.end(), later);
      const int64_t k = heap.back();
      heap.pop_back();
      order.push_back(k);
      for (int64_t j : succ[k])
        if (--indeg[j] == 0) {
          heap.push_back(j);
          std::push_heap(heap.begin(), heap.end(), later);
        }
    }
    // strands to warps, least loaded first (ties: lowest warp)
    std::vector<std::vector<int64_t>> wl(nwarps);
    std::vector<int64_t> load(nwarps, 0);
    for (int64_t k : order) {
      const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      wl[w].push_back(k);
      load[w] += sfirst[k + 1] - sfirst[k];
    }
    // tasks warp by warp; entries of the current task and of the strand's
    // previous task's last row become register-resolved markers
    for (int w = 0; w < NWARP; w++) {
      out.wptr[s * (NWARP + 1) + w] = (int32_t)(out.task.size() / 2);
      if (w >= nwarps) continue;
      for (int64_t k : wl[w])
        for (int64_t t = sfirst[k]; t < sfirst[k + 1]; t++) {
          const int64_t i0 = tfirst[t];
          const int cnt = tcnt[t];
          const int64_t prevlast = (t > sfirst[k]) ? row(i0 - 1) : -1;
          bool seq = false;
          for (int a = 0; a < cnt; a++) {
            const int64_t r = row(i0 + a);
            if (r >= n) continue;
            const int64_t base = E.off[s] + (r - b0) * E.width[s];
            int64_t slot = 0;
            // markers first (they must sit in the first entries of the row)
            for (int pass = 0; pass < 2; pass++)
              for (int64_t e = rp[r]; e < rp[r + 1]; e++) {
                const int64_t c = col[e];
                int d = 0;
                for (int a2 = 0; a2 < a; a2++)
                  if (row(i0 + a2) == c) d = a - a2;
                if (d == 0 && c == prevlast) d = a + 1;
                if ((pass == 0) != (d > 0)) continue;
                E.col[base + slot] = d > 0 ? -2 - d : (int32_t)c;
                E.val[base + slot] = TV(val[e]);
                slot++;
                if (d > 0 && d <= a) seq = true;
              }
          }
          out.task.push_back((int32_t)row(i0));
          out.task.push_back(cnt | (seq ? 8 : 0));
        }
    }
    out.wptr[s * (NWARP + 1) + NWARP] = (int32_t)(out.task.size() / 2);
    out.nstrands += nstr;
  }
}

template void build_chain<float>(const Permuted &, int64_t, bool, int, ChainHost<float> &);
template void build_chain<double>(const Permuted &, int64_t, bool, int, ChainHost<double> &);

void permute(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, const Factor &F,
             const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm, int64_t npad, Permuted &P) {
  P.n = n;
  P.npad = npad;
  P.lev.assign(n, 0);
  P.levU.assign(n, 0);
  for (int64_t i = 0; i < n; i++) {
    P.lev[i] = F.levL[perm[i]];
    P.levU[i] = F.levU[perm[i]];
  }
  // A' = P A P^T, rows sorted by new column
  std::vector<std::pair<int32_t, double>> tmp;
  P.Arp.assign(n + 1, 0);
  P.Acol.clear();
  P.Aval.clear();
  P.Acol.reserve(rp[n]);
  P.Aval.reserve(rp[n]);
  for (int64_t i = 0; i < n; i++) {
    const int64_t o = perm[i];
    tmp.clear();
    for (int64_t e = rp[o]; e < rp[o + 1]; e++) tmp.push_back({iperm[ci[e]], va[e]});
    std::sort(tmp.begin(), tmp.end(), [](auto &a, auto &b) { return a.first < b.first; });
    for (auto &t : tmp) {
      P.Acol.push_back(t.first);
      P.Aval.push_back(t.second);
    }
    P.Arp[i + 1] = (int64_t)P.Acol.size();
  }
  // strictly lower part of L' and strictly upper part of U' = L'^T, diagonal
  P.diag.assign(n, 0.0);
  P.Lrp.assign(n + 1, 0);
  P.Lcol.clear();
  P.Lval.clear();
  for (int64_t i = 0; i < n; i++) {
    const int64_t o = perm[i];
    tmp.clear();
    for (int64_t e = F.Lrowptr[o]; e < F.Lrowptr[o + 1]; e++) {
      if (F.Lcol[e] == o)
        P.diag[i] = F.Lval[e];
      else
        tmp.push_back({iperm[F.Lcol[e]], F.Lval[e]});
    }
    std::sort(tmp.begin(), tmp.end(), [](auto &a, auto &b) { return a.first < b.first; });
    for (auto &t : tmp) {
      P.Lcol.push_back(t.first);
      P.Lval.push_back(t.second);
    }
    P.Lrp[i + 1] = (int64_t)P.Lcol.size();
  }
  P.Urp.assign(n + 1, 0);
  P.Ucol.clear();
  P.Uval.clear();
  for (int64_t i = 0; i < n; i++) {
    const int64_t o = perm[i];  // row i of U' = column o of L
    tmp.clear();
    for (int64_t e = F.Ccolptr[o] + 1; e < F.Ccolptr[o + 1]; e++) tmp.push_back({iperm[F.Crow[e]], F.Cval[e]});
    std::sort(tmp.begin(), tmp.end(), [](auto &a, auto &b) { return a.first < b.first; });
    for (auto &t : tmp) {
      P.Ucol.push_back(t.first);
      P.Uval.push_back(t.second);
    }
    P.Urp[i + 1] = (int64_t)P.Ucol.size();
  }
}

}  // namespace nle
