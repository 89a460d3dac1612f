// Host-only test shim: runs the library's own host set-up code (the IC
// factor and the layouts of its triangular solves, nle_setup.cpp) without a
// GPU, so tests/test_chain_schedule.py can check the schedules on the CPU.
// Built by that test with g++; not part of the library.
#include <cstring>
#include <vector>

#include "../paper_1312_1553_gb300/csrc/nle_internal.h"
#include "../paper_1312_1553_gb300/csrc/nle_setup.h"

using namespace nle;

static Factor g_F;
static Permuted g_P;
static ChainHost<double> g_C[2];
static std::vector<int64_t> g_rp;
static std::vector<int32_t> g_ci;
static std::vector<double> g_va;
static Permuted g_PL;
static SellSet<double> g_S;
static std::vector<int32_t> g_perm;

extern "C" int shim_factor(int64_t n, const int64_t *rp, const int32_t *ci, const double *va, int lfil, double tau) {
  int64_t bad = -1;
  if (ic_factor_host(n, rp, ci, va, lfil, tau, g_F, &bad) != 0) return -1;
  g_rp.assign(rp, rp + n + 1);
  g_ci.assign(ci, ci + rp[n]);
  g_va.assign(va, va + rp[n]);
  std::vector<int32_t> perm(n), iperm(n);
  for (int64_t i = 0; i < n; i++) perm[i] = iperm[i] = (int32_t)i;
  const int64_t npad = (n + 127) / 128 * 128;
  permute(n, rp, ci, va, g_F, perm, iperm, npad, g_P);
  return 0;
}

// Build the chain schedule of L (lower = 1) or U (0); returns the number of
// tasks and the ELL size through *nent.
extern "C" int64_t shim_chain(int lower, int64_t bsize, int nwarps, int64_t *nent, int64_t *nslab) {
  ChainHost<double> &C = g_C[lower ? 1 : 0];
  build_chain<double>(g_P, bsize, lower != 0, nwarps, C);
  *nent = (int64_t)C.ell.col.size();
  *nslab = (int64_t)C.ell.width.size();
  return (int64_t)C.task.size() / 2;
}

extern "C" void shim_chain_get(int lower, int64_t *off, int32_t *width, int32_t *col, double *val, int32_t *wptr,
                               int32_t *task, double *diag) {
  ChainHost<double> &C = g_C[lower ? 1 : 0];
  memcpy(off, C.ell.off.data(), C.ell.off.size() * 8);
  memcpy(width, C.ell.width.data(), C.ell.width.size() * 4);
  memcpy(col, C.ell.col.data(), C.ell.col.size() * 4);
  memcpy(val, C.ell.val.data(), C.ell.val.size() * 8);
  memcpy(wptr, C.wptr.data(), C.wptr.size() * 4);
  memcpy(task, C.task.data(), C.task.size() * 4);
  memcpy(diag, g_P.diag.data(), g_P.diag.size() * 8);
}

// Level schedule layout: slab-major level-minor relabelling, per-slab ELL of
// L and U with the rounds of every group of R rows; *nent: the ELL size of L
// (lower = 1) or U.  Returns npad.
extern "C" int64_t shim_level(int lower, int64_t bsize, int R, int64_t *nent, int64_t *nslab) {
  const int64_t n = g_F.n;
  const int64_t npad = (n + 127) / 128 * 128;
  std::vector<int32_t> iperm;
  slab_level_order(g_F, bsize, nullptr, g_perm, iperm);
  permute(n, g_rp.data(), g_ci.data(), g_va.data(), g_F, g_perm, iperm, npad, g_PL);
  build_sell<double>(g_PL, 128, bsize, false, R, g_S);
  *nent = (int64_t)(lower ? g_S.L.col.size() : g_S.U.col.size());
  *nslab = (int64_t)g_S.L.width.size();
  return npad;
}

extern "C" void shim_level_get(int lower, int64_t *off, int32_t *width, int32_t *col, double *val, uint16_t *round,
                               double *rdiag, int32_t *perm) {
  const EllHost<double> &E = lower ? g_S.L : g_S.U;
  memcpy(off, E.off.data(), E.off.size() * 8);
  memcpy(width, E.width.data(), E.width.size() * 4);
  memcpy(col, E.col.data(), E.col.size() * 4);
  memcpy(val, E.val.data(), E.val.size() * 8);
  memcpy(round, E.round.data(), E.round.size() * 2);
  memcpy(rdiag, g_S.diag.data(), g_S.diag.size() * 8);
  memcpy(perm, g_perm.data(), g_perm.size() * 4);
}
