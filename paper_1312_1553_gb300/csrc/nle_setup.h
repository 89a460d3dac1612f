// Host-side set-up of the nle library (see nle_setup.cpp).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace nle {

struct Factor {
  int64_t n = 0;
  // L by rows, diagonal last (exported by nle_get_factor)
  std::vector<int64_t> Lrowptr;
  std::vector<int32_t> Lcol;
  std::vector<double> Lval;
  // L by columns, diagonal first (= U = L^T by rows)
  std::vector<int64_t> Ccolptr;
  std::vector<int32_t> Crow;
  std::vector<double> Cval;
  std::vector<int32_t> levL, levU;
  int64_t nlevL = 0, nlevU = 0;
};

// Relabelled (slab-major, level-minor) matrices, row by row.
struct Permuted {
  int64_t n = 0, npad = 0;
  std::vector<int64_t> Arp, Lrp, Urp;
  std::vector<int32_t> Acol, Lcol, Ucol;
  std::vector<double> Aval, Lval, Uval, diag;
  std::vector<int32_t> lev;   // level (of L) of every relabelled row
  std::vector<int32_t> levU;  // level (of U = L^T) of every relabelled row
};

template <typename TV>
struct SellHost {
  int64_t nslices = 0;
  std::vector<int64_t> sptr;
  std::vector<int32_t> col;
  std::vector<TV> val;
};

// Strictly triangular part in per-slab ELL form (see trsv_block).
template <typename TV>
struct EllHost {
  std::vector<int64_t> off;    // per slab: first entry
  std::vector<int32_t> width;  // per slab: entries per row, multiple of 8
  std::vector<int32_t> col;    // -1 = padding
  std::vector<TV> val;
  // per row (level schedule): bits 0-3 its round inside its group of R
  // rows, bits 4-7 the group's last round, bits 8-15 the group's overflow
  // steps (entries past the 2 * 32 / R a warp step prefetches, in steps of
  // 32 / R; 255: up to the slab's width)
  std::vector<uint16_t> round;
};

// Chain schedule of one strictly triangular factor (see trsv_chain): the
// rows of each slab are cut into tasks of at most TRSV_ROWS consecutive rows
// (in processing order: ascending for L, descending for U); consecutive tasks
// whose first row depends on the previous task's last row form a strand,
// which one warp solves task after task with that dependency held in
// registers.  Strands are dealt to the warps of the slab's CTA in a
// topological order of the strand graph, so every wait ends.
template <typename TV>
struct ChainHost {
  EllHost<TV> ell;            // per-slab ELL; an entry resolved in registers carries col = -2 - d,
                              // d = distance back in the warp's processing order (1..TRSV_ROWS)
  std::vector<int32_t> wptr;  // per slab: NWARP + 1 offsets into task (warp w: [wptr[w], wptr[w+1]))
  std::vector<int32_t> task;  // per task: first row processed, rows | (sequential ? 8 : 0)
  int64_t nstrands = 0;
};

template <typename TV>
struct SellSet {
  SellHost<TV> A;
  SellHost<double> A64;
  EllHost<TV> L, U;      // strictly lower / upper parts, slab-major order
  std::vector<TV> diag;  // npad: reciprocal pivots 1 / L_ii, 1 on padding rows
};

// 0 on success; 2 = malformed CSR, 3 = non-positive diagonal (msg says why).
int validate_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci, const double *va, std::string &msg);

// IC(lfil, tau) of A plus the levels of L and L^T.  0 on success, -2 on a
// non-positive pivot (column in *bad_col).
int ic_factor_host(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, int lfil, double tau,
                   Factor &F, int64_t *bad_col);
// The factor from L by columns (column k: entries cs[k]..cs[k+1]-1 of
// rows/vals, diagonal first, rows ascending): L by rows and the levels.
void factor_from_columns(int64_t n, std::vector<int64_t> cs, std::vector<int32_t> rows, std::vector<double> vals,
                         Factor &F);

// Greedy multicolour ordering (nle_multicolor_order in nle.h): perm[new] =
// old, rows by colour then by row.  Returns the number of colours.
int32_t multicolor_order(int64_t n, const int64_t *rp, const int32_t *ci, int distance, std::vector<int32_t> &perm);
// B = P A P^T (perm[new] = old) in CSR with ascending columns in every row.
void permute_csr(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, const std::vector<int32_t> &perm,
                 std::vector<int64_t> &brp, std::vector<int32_t> &bci, std::vector<double> &bva);
// perm[new] = old: rows cut into slabs of bsize consecutive values of
// locality[row] (the row itself when locality is NULL; locality must be a
// permutation of 0..n-1); inside a slab, by level of L, then by locality.
// P L P^T stays lower triangular.
void slab_level_order(const Factor &F, int64_t bsize, const int32_t *locality, std::vector<int32_t> &perm,
                      std::vector<int32_t> &iperm);

void permute(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, const Factor &F,
             const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm, int64_t npad, Permuted &P);

// level_rounds: split every group of R rows (the rows a warp of the level
// schedule takes at a time, 4 or 2) into one round per level (needed when
// dependencies can point to later slabs; see trsv_block).
template <typename TV>
void build_sell(const Permuted &P, int H, int64_t bsize, bool level_rounds, int R, SellSet<TV> &S);

// Chain schedule of the strictly lower (lower = true: P.Lrp/Lcol/Lval, levels
// P.lev) or upper (P.Urp/Ucol/Uval, levels P.levU) factor for nwarps warps
// per slab.  Needs the identity relabelling (slabs are ranges of the
// factored matrix's own row order).
template <typename TV>
void build_chain(const Permuted &P, int64_t bsize, bool lower, int nwarps, ChainHost<TV> &out);

}  // namespace nle
