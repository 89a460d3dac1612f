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
  return 0;
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
// order), plus the round of every row inside its group of TRSV_ROWS rows: the length
// of the longest dependency chain ending at the row within the group
// (lower: earlier rows of the group; upper: later rows).
template <typename TV>
static void ell(int64_t n, int64_t npad, int64_t bsize, bool lower, const std::vector<int64_t> &rp,
                const std::vector<int32_t> &col, const std::vector<double> &val, const std::vector<int32_t> *lev,
                EllHost<TV> &out) {
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
  for (int64_t g0 = 0; g0 < n; g0 += TRSV_ROWS) {
    const int64_t g1 = std::min(n, g0 + TRSV_ROWS);
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
        out.round[r] = (uint8_t)rank;
      }
    } else if (lower) {
      for (int64_t r = g0; r < g1; r++)
        for (int64_t e = rp[r]; e < rp[r + 1]; e++)
          if (col[e] >= g0) out.round[r] = std::max<uint8_t>(out.round[r], out.round[col[e]] + 1);
    } else {
      for (int64_t r = g1 - 1; r >= g0; r--)
        for (int64_t e = rp[r]; e < rp[r + 1]; e++)
          if (col[e] < g1) out.round[r] = std::max<uint8_t>(out.round[r], out.round[col[e]] + 1);
    }
  }
}

template <typename TV>
void build_sell(const Permuted &P, int H, int64_t bsize, bool level_rounds, SellSet<TV> &S) {
  pack<TV>(P.n, P.npad, H, P.Arp, P.Acol, P.Aval, 0, 0, S.A);
  pack<double>(P.n, P.npad, H, P.Arp, P.Acol, P.Aval, 0, 0, S.A64);
  const std::vector<int32_t> *lev = level_rounds ? &P.lev : nullptr;
  ell<TV>(P.n, P.npad, bsize, true, P.Lrp, P.Lcol, P.Lval, lev, S.L);
  ell<TV>(P.n, P.npad, bsize, false, P.Urp, P.Ucol, P.Uval, lev, S.U);
  S.diag.assign(P.npad, TV(1));
  for (int64_t i = 0; i < P.n; i++) S.diag[i] = TV(1.0 / P.diag[i]);  // reciprocal pivots
}

template void build_sell<float>(const Permuted &, int, int64_t, bool, SellSet<float> &);
template void build_sell<double>(const Permuted &, int, int64_t, bool, SellSet<double> &);

void permute(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, const Factor &F,
             const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm, int64_t npad, Permuted &P) {
  P.n = n;
  P.npad = npad;
  P.lev.assign(n, 0);
  for (int64_t i = 0; i < n; i++) P.lev[i] = F.levL[perm[i]];
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
