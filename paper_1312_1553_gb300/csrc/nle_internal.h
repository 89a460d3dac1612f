// Internal data structures of the nle library (host setup + CUDA kernels).
//
// Layout in HBM
//   Every device vector and matrix is stored in SLAB-MAJOR, LEVEL-MINOR
//   order: the rows are cut into one slab per CTA (bsize consecutive rows of
//   the caller's order) and sorted by their level in the IC factor L inside
//   each slab; position i holds the caller's row perm[i].  Relabelling the
//   unknowns changes no arithmetic of the method (dot products are
//   permutation invariant and P L P^T stays triangular because a row only
//   depends on rows of lower level), but every CTA then solves a contiguous
//   range of rows.  Vectors are padded to npad (a multiple of the slice
//   height) with zeros.
//
//   A uses a sliced-ELL format ("SELL") with slice height H = 32 * VW rows,
//   where VW = 16 / sizeof(T) consecutive rows belong to one thread: a warp
//   owns one slice, a lane owns VW adjacent rows and loads their e-th entries
//   with one 16-byte load (val[base + e*H + lane*VW + v]); padding entries
//   carry value 0 and column = the row itself.  The strictly triangular
//   parts of L and L^T are stored per slab in ELL form (entries of a row
//   contiguous, column -1 for padding).
#pragma once
#include <cstdint>

#include <vector_types.h>

namespace nle {

constexpr int TPB = 512;         // threads per CTA of the persistent kernels
constexpr int NWARP = TPB / 32;  // warps per CTA
constexpr int KMAX = 10;         // largest k_max
constexpr int MMAX = 64;         // largest p (columns of Q)
constexpr int RED_MAX = 160;     // reduction slots per pass
// triangular solves: rows a warp takes at a time (4 or 8); lanes per row;
// entries per lane fetched ahead (16 per row)
#ifndef NLE_TRSV_ROWS
#define NLE_TRSV_ROWS 4
#endif
constexpr int TRSV_ROWS = NLE_TRSV_ROWS;
constexpr int TRSV_LANES = 32 / TRSV_ROWS;
constexpr int TRSV_EPL = 16 / TRSV_LANES;
static_assert(TRSV_ROWS == 4 || TRSV_ROWS == 8, "4 or 8 rows per warp");

template <typename T>
struct Sell {
  int64_t nslices = 0;
  const int64_t *sptr = nullptr;  // nslices+1 offsets (elements)
  const int32_t *col = nullptr;
  const T *val = nullptr;
};

// Persistent solver state in device memory.  Written by CTA 0 only, at
// points separated from every reader by a grid barrier or a kernel boundary.
struct State {
  int j;                 // eigenpair being computed (0-based)
  int k;                 // number of stored BFGS pairs
  int order[KMAX];       // chronological pair index -> physical slot
  double alpha[KMAX];    // s^T r of each stored pair (chronological)
  double theta;          // current Rayleigh quotient
  double rnorm;          // ||A u - theta u||
  int newton_its;
  // per eigenpair results
  double lambda[MMAX];
  double res[MMAX];
  int dacg_its[MMAX];
  int outer_its[MMAX];
  int pcg_its[MMAX];
  int conv[MMAX];
  long long mvp_dacg;
  long long mvp_newton;
  long long pcg_total;
  long long pcg_sum_m;   // sum over inner iterations of the columns of Q
  long long pcg_sum_k;   // sum over inner iterations of the stored pairs
  long long dacg_sum_m;  // sum over DACG iterations of the deflated columns
  long long dacg_total;  // DACG iterations
  int exits[5];
  double sign[MMAX];  // sign applied to each output eigenvector (largest entry positive)
  int adj_refine, adj_inner;  // refinement steps and inner iterations of the last adjoint solve
  double adj_res;             // its final relative FP64 residual
  // last single inner solve (nle_pcg)
  int last_its, last_exit;
  double last_g0, last_gn, last_eres;
  // error word (0 = ok, else nle_status) and where a wait gave up
  int err;
  int err_where;
  unsigned bar;  // grid barrier counter
  unsigned qf, qb;  // work queues (slices) of the forward / backward solve
  long long tphase[8];  // device time per phase (ns, measured by CTA 0)
};

struct Opts {
  double tol;
  double tau_pcg;
  double tau_dacg;
  int max_newton;
  int max_pcg;
  int max_dacg;
  int kmax;
  int exit_eigres;
  int exit_stag;
  int recompute;
  long long spin_ns;
  int trsv_warps;     // warps per CTA that take part in the triangular solves
  int poll_ns;        // pause between two polls of a triangular-solve wait (0: none)
  int bfgs_full;      // 1: pairs (s_k, r_k - r_{k+1}) (full BFGS update), 0: (s_k, r_k)
};

// Pointers handed to the persistent kernels (by value).
template <typename T>
struct Dev {
  int64_t n = 0;        // true size
  int64_t npad = 0;     // padded size (multiple of 32*VW)
  int64_t nchunks = 0;  // npad / VW
  int ldq = 0;          // allocated columns of Q / Qt
  int64_t bsize = 0;    // rows per CTA slab in the triangular solves (multiple of TRSV_ROWS)
  Sell<T> A;            // A in working precision
  Sell<double> A64;     // A in FP64 (same pattern and layout as A)
  // strictly lower part of L and strictly upper part of U = L^T in the
  // slab-major order, ELL per slab (offset and width per slab, col -1 =
  // padding), diagonal separate, and the round of every row in its group of TRSV_ROWS rows
  const int64_t *Loff = nullptr, *Uoff = nullptr;
  const int32_t *Lw = nullptr, *Uw = nullptr, *Lcol = nullptr, *Ucol = nullptr;
  const T *Lval = nullptr, *Uval = nullptr;
  const T *rdiag = nullptr;  // reciprocal diagonal of L (1 on padding rows)
  const uint16_t *Lround = nullptr, *Uround = nullptr;
  int trows = TRSV_ROWS;  // level schedule: rows a warp takes at a time (4, or 2 for wide rows)
  // chain schedule (chain = 1): the device order is the factored matrix's
  // own row order, and each slab's rows are solved as per-warp task lists
  // (Lwp/Uwp: NWARP + 1 offsets per slab into Ltask/Utask, a task = {first
  // row processed, rows | sequential << 3}); the ELL arrays above then hold
  // register-resolved entries as col = -2 - d (see trsv_chain)
  int chain = 0;
  const int32_t *Lwp = nullptr, *Uwp = nullptr;
  const int2 *Ltask = nullptr, *Utask = nullptr;
  // working-precision vectors (npad; z and c0 have npad + 32*VW entries)
  T *p, *y, *s, *g, *z, *c0, *rT, *x, *Ax, *Ap;
  const T *X0 = nullptr;  // optional: start vectors (p columns, device order) for the whole-solve kernel
  int grid = 0;           // CTAs this problem's layout was built for (slabs)
  T *Q;        // npad * ldq, column c at Q + c*npad (converged v_1.. and u)
  T *S, *R;    // npad * KMAX, BFGS pairs by physical slot
  // FP64 vectors
  double *u, *Au, *r, *t;
  double *y64, *b64;  // adjoint solve: solution and right-hand side
  double *Qt;  // npad * ldq, FP64 converged eigenvectors
  // reductions / control
  double *part;  // 2 * RED_MAX * gridDim
  State *st;
};

// Batched solve: problems taken from a device work queue by groups of G CTAs.
template <typename T>
struct Batch {
  const Dev<T> *devs;  // per problem
  const int *order;    // problems, largest first
  int count;
  int G;               // CTAs per group (every problem's layout uses <= G)
  int p;               // eigenpairs per problem
  unsigned *queue;     // next index into order
  unsigned *gbar;      // per group: barrier counter
  int *gslot;          // per group: index taken by the group
  int *gerr;           // per group: error word of the group barrier
  long long group_spin_ns;
};

}  // namespace nle
